"""FP64 CPU oracle of the simplified wall-modeled IBM stress stage (Sec. 3 of
Liu & Stevens, arXiv:2006.03343).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
The arithmetic lives in ``wmibm_oracle.c`` (plain C, double precision, loops in
the paper's order); this module compiles it with gcc and marshals numpy arrays.
The pseudo-spectral derivatives of Eqs. 13-14 are written here with numpy's FP64
FFT as the library step: a 2-D transform of each z-plane, exactly as the sum over
(k_x, k_y) is stated.  The Smagorinsky stress (Eqs. 4-7) is plain numpy as well.

Functions and the passages they follow:
  classify      Sec. 3.3, node classes on the w-grid and the uv-grid
  normals       Sec. 3.1, n = grad(phi)/|grad(phi)| (Eq. 24)
  interp        Sec. 3.3, second-order accurate interpolation (trilinear)
  wall_stress   Sec. 3.3, Eq. 28 and the tensor rotation tau_ij = a_im a_jn tau'_mn
  wall_model_node  the same wall model evaluated at a single node
  force         Eq. 2 / Eq. 18: f = -div(tau) on the staggered grid (Eqs. 15-16)
  horizontal_derivatives  Eqs. 13-14, pseudo-spectral d/dx and d/dy of one field
  force_spectral  f = -div(tau) with the horizontal derivatives of Eqs. 13-14
  sgs_stress    Eqs. 4-7, the Smagorinsky stress with Mason's wall damping at fluid nodes
  mask          Sec. 3.2, Eq. 27: the body velocity condition
  adjoint       chain rule of wall_stress + force for L = <g, f>
  heightfield_distance  Sec. 3.1, d = the minimum distance to the immersed boundary, for
                a height field's piecewise-linear surface (reading R10), by brute force
  heightfield_sdf  Sec. 3.1, phi = +d in the fluid, -d in the solid, within a reach

Every function here is pinned against closed forms, invariants and brute force
(see the docstrings there): ``tests/test_oracle_pins.py`` (wall stress, central-
difference divergence, mask), ``tests/test_oracle_adjoint.py`` (adjoint) and
``tests/test_oracle_spectral.py`` (pseudo-spectral divergence),
``tests/test_oracle_sgs.py`` (Smagorinsky stress) and ``tests/test_oracle_sdf.py``
(height-field distance).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wmibm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP for the loops marked so)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.orc_classify.argtypes = [_I64, _I64, _I64, _D, _D, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_normals.argtypes = [_I64, _I64, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    _D, _D]
        lib.orc_interp.argtypes = [_I64, _I64, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   _D, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.orc_interp.restype = ctypes.c_double
        lib.orc_wall_stress.argtypes = ([_I64, _I64, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         _D, _D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _D, _D, _D] + [_D] * 6 + [_D])
        lib.orc_wall_stress.restype = ctypes.c_int
        lib.orc_wall_model_node.argtypes = [_I64, _I64, _I64, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, _D, ctypes.c_int, _I64, _I64, _I64,
                                            _D, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            _D, _D]
        lib.orc_force.argtypes = [_I64, _I64, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double] + [_D] * 9
        lib.orc_mask.argtypes = [_I64, _I64, _I64, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_double]
        lib.orc_force_adjoint.argtypes = [_I64, _I64, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          _D, _D, _D, _D, _D, _D, _D, _D, _D]
        lib.orc_force_adjoint.restype = None
        if hasattr(lib, "orc_adjoint"):
            lib.orc_adjoint.argtypes = ([_I64, _I64, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         _D, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         _D, _D, _D, _D, _D, _D, _D, _D, _D, _D])
            lib.orc_adjoint.restype = ctypes.c_int
        lib.orc_heightfield_distance.argtypes = [_I64, _I64, _I64, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, _D, _I64, ctypes.c_void_p, ctypes.c_int, _D]
        lib.orc_heightfield_distance.restype = None
        lib.orc_openmp_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle takes C-contiguous float64 arrays"
    return a.ctypes.data_as(_D)


def _shape(grid):
    nx, ny, nz, lx, ly, lz = grid
    return int(nx), int(ny), int(nz), float(lx), float(ly), float(lz)


def openmp_threads() -> int:
    return int(_load().orc_openmp_threads())


def set_threads(n: int) -> None:
    """Thread count of the oracle's parallel loops (for timing; results do not depend on it)."""
    _load().orc_set_threads(int(n))


def classify(grid, phi_uv, phi_w, phi_b):
    """Sec. 3.3 classes per node: 0 fluid, 1 band, 2 solid -> (cls_uv, cls_w) int8 arrays."""
    nx, ny, nz, *_ = _shape(grid)
    cu = np.empty(phi_uv.shape, np.int8)
    cw = np.empty(phi_w.shape, np.int8)
    _load().orc_classify(nx, ny, nz, _p(phi_uv), _p(phi_w), float(phi_b),
                         cu.ctypes.data_as(ctypes.c_void_p), cw.ctypes.data_as(ctypes.c_void_p))
    return cu, cw


def normals(grid, phi):
    """Sec. 3.1 unit normals on phi's own grid -> array [3, nz, ny, nx]."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    out = np.empty((3,) + phi.shape, np.float64)
    _load().orc_normals(nx, ny, nz, lx, ly, lz, _p(phi), _p(out))
    return out


def interp(grid, f, is_w, x, y, z):
    nx, ny, nz, lx, ly, lz = _shape(grid)
    return float(_load().orc_interp(nx, ny, nz, lx, ly, lz, _p(f), int(is_w), float(x), float(y), float(z)))


def wall_stress(grid, phi_uv, phi_w, z0, phi_c, phi_b, u, v, w, tau, kappa=0.4, logz0=None):
    """Sec. 3.3 wall stress.  tau: dict of 6 float64 arrays (txx txy tyy tzz txz tyz),
    updated in place.  z0: float or per-cell array; or logz0: per-cell ln z0 (then
    C = kappa^2 / (ln phi_c - ln z0)^2 and z0 is ignored).  Returns stats [2, 6]:
    rows (w-band, uv-band), columns (count, sum tau_w, sum tau_w^2, min tau_w, max U_r,
    nodes whose sample point x_c lies outside the physical levels of the uv-grid or the
    w-grid, where the interpolation clamps it: reading R3)."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    if logz0 is not None:
        z0a = np.ascontiguousarray(logz0, np.float64)
        is_field = 2
    elif np.isscalar(z0):
        z0a = np.array([float(z0)], np.float64)
        is_field = 0
    else:
        z0a = np.ascontiguousarray(z0, np.float64)
        is_field = 1
    stats = np.zeros(12, np.float64)
    rc = _load().orc_wall_stress(nx, ny, nz, lx, ly, lz, _p(phi_uv), _p(phi_w), _p(z0a), is_field,
                                 float(phi_c), float(kappa), float(phi_b), _p(u), _p(v), _p(w),
                                 _p(tau["txx"]), _p(tau["txy"]), _p(tau["tyy"]), _p(tau["tzz"]),
                                 _p(tau["txz"]), _p(tau["tyz"]), _p(stats))
    if rc == -2:
        raise MemoryError("oracle: out of memory in the wall-stress pass")
    if rc != 0:
        raise ValueError("oracle: z0 must satisfy 0 < z0 < phi_c")
    return stats.reshape(2, 6)


def wall_model_node(grid, phi, is_w, i, j, k, u, v, w, z0, phi_c, kappa=0.4):
    """The Sec. 3.3 wall model at one node -> (tau 3x3, tau_w, |U_r|)."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    t9 = np.zeros(9, np.float64)
    tw = np.zeros(2, np.float64)
    _load().orc_wall_model_node(nx, ny, nz, lx, ly, lz, _p(phi), int(is_w), int(i), int(j), int(k),
                                _p(u), _p(v), _p(w), float(z0), float(phi_c), float(kappa), _p(t9), _p(tw))
    return t9.reshape(3, 3), float(tw[0]), float(tw[1])


def force(grid, tau):
    """f = -div(tau) (Eq. 2, Eqs. 15-16, central differences in x and y) -> (fx, fy, fz)."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    shp = tau["txx"].shape
    fx, fy, fz = (np.empty(shp, np.float64) for _ in range(3))
    _load().orc_force(nx, ny, nz, lx, ly, lz, _p(tau["txx"]), _p(tau["txy"]), _p(tau["tyy"]),
                      _p(tau["tzz"]), _p(tau["txz"]), _p(tau["tyz"]), _p(fx), _p(fy), _p(fz))
    return fx, fy, fz


def wavenumbers(n, length):
    """Wavenumbers of an n-point periodic direction of length L (Eqs. 13-14):
    k_m = 2 pi m / L with m = 0, 1, ..., then negative m from the top of the range.
    For even n the Nyquist mode m = n/2 is given k = 0: i k A for it would not be
    the transform of a real field, so it carries no first derivative."""
    m = np.arange(n)
    m = np.where(m < (n + 1) // 2, m, m - n).astype(np.float64)
    if n % 2 == 0:
        m[n // 2] = 0.0
    return 2.0 * np.pi * m / float(length)


def horizontal_derivatives(grid, a):
    """Eqs. 13-14 for one field a[k][j][i]: per z-plane the Fourier amplitudes
    A(k_x, k_y) (2-D FFT divided by nx ny), then the sums over (k_x, k_y) of
    i k_x A e^{i(k_x x + k_y y)} and i k_y A e^{i(k_x x + k_y y)} -> (da/dx, da/dy)."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    amp = np.fft.fft2(np.asarray(a, np.float64), axes=(1, 2)) / (nx * ny)
    kx = wavenumbers(nx, lx)[None, None, :]
    ky = wavenumbers(ny, ly)[None, :, None]
    # ifft2 divides by nx ny; the synthesis sum does not
    ddx = np.fft.ifft2(1j * kx * amp, axes=(1, 2)) * (nx * ny)
    ddy = np.fft.ifft2(1j * ky * amp, axes=(1, 2)) * (nx * ny)
    return np.ascontiguousarray(ddx.real), np.ascontiguousarray(ddy.real)


def force_spectral(grid, tau):
    """f = -div(tau) (Eq. 2 / Eq. 18) with the paper's own horizontal scheme: x and y
    derivatives pseudo-spectral (Eqs. 13-14), vertical ones the staggered differences
    of Eqs. 15-16.  f_x, f_y sit on uv-levels and take (t_.z[k+1] - t_.z[k]) / dz of the
    w-level stresses; f_z sits on w-levels and takes (tzz[k] - tzz[k-1]) / dz.
    f_x = f_y = 0 on the ghost uv-level nz-1; f_z = 0 on the floor and the lid.
    -> (fx, fy, fz)."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    dz = lz / (nz - 1)
    t = {k: np.asarray(v, np.float64) for k, v in tau.items()}
    dxx_dx, _ = horizontal_derivatives(grid, t["txx"])
    dxy_dx, dxy_dy = horizontal_derivatives(grid, t["txy"])
    _, dyy_dy = horizontal_derivatives(grid, t["tyy"])
    dxz_dx, _ = horizontal_derivatives(grid, t["txz"])
    _, dyz_dy = horizontal_derivatives(grid, t["tyz"])
    shp = t["txx"].shape
    fx, fy, fz = (np.zeros(shp, np.float64) for _ in range(3))
    fx[:-1] = -(dxx_dx[:-1] + dxy_dy[:-1] + (t["txz"][1:] - t["txz"][:-1]) / dz)
    fy[:-1] = -(dxy_dx[:-1] + dyy_dy[:-1] + (t["tyz"][1:] - t["tyz"][:-1]) / dz)
    fz[1:-1] = -(dxz_dx[1:-1] + dyz_dy[1:-1] + (t["tzz"][1:-1] - t["tzz"][:-2]) / dz)
    return fx, fy, fz


def _ddx(q, h):
    """Periodic central difference along x (the last axis)."""
    return (np.roll(q, -1, axis=2) - np.roll(q, 1, axis=2)) / (2.0 * h)


def _ddy(q, h):
    """Periodic central difference along y (the middle axis)."""
    return (np.roll(q, -1, axis=1) - np.roll(q, 1, axis=1)) / (2.0 * h)


def mixing_length_sq(phi, z0, cs, kappa, grid):
    """Eq. 7 with n = 2: 1/lambda^2 = 1/lambda_0^2 + 1/[kappa (z + z0)]^2 with
    lambda_0 = C_s l, l = (dx dy dz)^(1/3) (Eq. 6), and z the node's distance phi
    above the surface -> lambda^2."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    ell = (lx / nx * ly / ny * lz / (nz - 1)) ** (1.0 / 3.0)
    lam0 = cs * ell
    return 1.0 / (1.0 / lam0 ** 2 + 1.0 / (kappa * (phi + z0)) ** 2)


def sgs_stress(grid, phi_uv, phi_w, z0, phi_b, u, v, w, tau, cs=0.16, kappa=0.4):
    """Smagorinsky stress (Eqs. 4-7) written into tau (dict of 6 arrays) at fluid nodes.

    tau_ij = -2 nu_t S_ij, S = (grad u + grad u^T)/2, nu_t = lambda^2 |S|,
    |S| = sqrt(2 S:S), lambda from mixing_length_sq (Mason's damping, z -> phi).
    Each component sits on its own node: S11, S22, S12, S33 on uv-nodes (S33 from
    the w-levels above and below, Eq. 16), S13, S23 on w-nodes (the z-derivative of
    u, v from the uv-levels below and above, Eq. 15); x, y derivatives are periodic
    central differences.  |S| on a uv-node averages S13, S23 of the w-levels below
    and above it; on a w-node it averages S11, S22, S33, S12 of the uv-levels below
    and above it.  At the floor w-level S13, S23 repeat those of the level above;
    at the lid they are 0 (no stress there, Eq. 10); both enter only that average.  Fluid nodes are those of neither the band nor
    the solid class (Sec. 3.3); band and solid entries, the ghost uv-level and the
    floor w-level keep their values; at the lid w-level tau_xz = tau_yz = 0
    (Eq. 10).  z0: scalar or per-cell array."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    dx, dy, dz = lx / nx, ly / ny, lz / (nz - 1)
    u, v, w = (np.asarray(a, np.float64) for a in (u, v, w))
    S11 = _ddx(u, dx)
    S22 = _ddy(v, dy)
    S12 = 0.5 * (_ddy(u, dy) + _ddx(v, dx))
    S33 = np.zeros_like(u)
    S33[:-1] = (w[1:] - w[:-1]) / dz
    S13 = np.zeros_like(u)
    S23 = np.zeros_like(u)
    S13[1:-1] = 0.5 * ((u[1:-1] - u[:-2]) / dz + _ddx(w, dx)[1:-1])
    S23[1:-1] = 0.5 * ((v[1:-1] - v[:-2]) / dz + _ddy(w, dy)[1:-1])
    S13[0], S23[0] = S13[1], S23[1]
    # |S| on uv-levels 0 .. nz-2 and on w-levels 1 .. nz-2
    s13u = 0.5 * (S13[:-1] + S13[1:])
    s23u = 0.5 * (S23[:-1] + S23[1:])
    mag_uv = np.sqrt(2.0 * (S11[:-1] ** 2 + S22[:-1] ** 2 + S33[:-1] ** 2)
                     + 4.0 * (S12[:-1] ** 2 + s13u ** 2 + s23u ** 2))
    avg = lambda q: 0.5 * (q[:-2] + q[1:-1])          # uv-levels k-1 and k for w-levels k = 1 .. nz-2
    mag_w = np.sqrt(2.0 * (avg(S11) ** 2 + avg(S22) ** 2 + avg(S33) ** 2)
                    + 4.0 * (avg(S12) ** 2 + S13[1:-1] ** 2 + S23[1:-1] ** 2))
    z0a = z0 if np.isscalar(z0) else np.asarray(z0, np.float64)
    lam_uv = mixing_length_sq(np.asarray(phi_uv, np.float64), z0a, cs, kappa, grid)
    lam_w = mixing_length_sq(np.asarray(phi_w, np.float64), z0a, cs, kappa, grid)
    cls_uv, cls_w = classify(grid, phi_uv, phi_w, phi_b)
    fl_uv = cls_uv[:-1] == 0
    nu_uv = lam_uv[:-1] * mag_uv
    for name, S in (("txx", S11), ("tyy", S22), ("tzz", S33), ("txy", S12)):
        t = tau[name][:-1]
        t[fl_uv] = (-2.0 * nu_uv * S[:-1])[fl_uv]
    fl_w = cls_w[1:-1] == 0
    nu_w = lam_w[1:-1] * mag_w
    for name, S in (("txz", S13), ("tyz", S23)):
        t = tau[name][1:-1]
        t[fl_w] = (-2.0 * nu_w * S[1:-1])[fl_w]
        lid = tau[name][-1]
        lid[cls_w[-1] == 0] = 0.0
    return tau


def mask(grid, phi_uv, phi_w, u, v, w, gradp=None, dt=0.0):
    """Eq. 27 in place on (u, v, w); gradp = (dp/dx, dp/dy, dp/dz) on the velocity grids or None."""
    nx, ny, nz, *_ = _shape(grid)
    gx, gy, gz = gradp if gradp is not None else (None, None, None)
    _load().orc_mask(nx, ny, nz, _p(phi_uv), _p(phi_w), _p(u), _p(v), _p(w), _p(gx), _p(gy), _p(gz), float(dt))


def force_adjoint(grid, g):
    """Transpose of force(): dL/dtau for L = sum(g . f), g = (gx, gy, gz) -> dict of 6 arrays."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    shp = g[0].shape
    out = {k: np.empty(shp, np.float64) for k in ("txx", "txy", "tyy", "tzz", "txz", "tyz")}
    _load().orc_force_adjoint(nx, ny, nz, lx, ly, lz, _p(g[0]), _p(g[1]), _p(g[2]), _p(out["txx"]),
                              _p(out["txy"]), _p(out["tyy"]), _p(out["tzz"]), _p(out["txz"]), _p(out["tyz"]))
    return out


def adjoint(grid, phi_uv, phi_w, logz0, phi_c, phi_b, u, v, w, g, kappa=0.4):
    """Hand-derived adjoint of one stage (wall stress with per-cell ln z0, then f = -div tau)
    for L = sum(g . f) -> (du, dv, dw, dlogz0)."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    shp = u.shape
    du, dv, dw, ds = (np.empty(shp, np.float64) for _ in range(4))
    rc = _load().orc_adjoint(nx, ny, nz, lx, ly, lz, _p(phi_uv), _p(phi_w), _p(np.ascontiguousarray(logz0)),
                             float(phi_c), float(kappa), float(phi_b), _p(u), _p(v), _p(w),
                             _p(g[0]), _p(g[1]), _p(g[2]), _p(du), _p(dv), _p(dw), _p(ds))
    if rc == -1:
        raise ValueError("oracle: every z0 = exp(logz0) must satisfy 0 < z0 < phi_c")
    if rc != 0:
        raise MemoryError("oracle: no scratch memory for the adjoint")
    return du, dv, dw, ds


def heightfield_distance(grid, h2d, is_w, nodes=None):
    """Sec. 3.1: d = the minimum distance from a node to the immersed boundary, here
    the piecewise-linear surface through the heights h2d[ny, nx] sampled at the
    column nodes (reading R10: each cell split along its (i, j)-(i+1, j+1)
    diagonal), by brute force over every triangle.  Returns d for every node of
    the uv-grid (is_w False) or the w-grid (is_w True) as [nz, ny, nx], or at the
    flat indices `nodes`.  Only distances below half the period minus a cell are
    exact (each triangle is taken at its periodic image nearest the node)."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    hh = np.ascontiguousarray(h2d, dtype=np.float64)
    assert hh.shape == (ny, nx)
    if nodes is None:
        out = np.empty((nz, ny, nx))
        _load().orc_heightfield_distance(nx, ny, nz, lx, ly, lz, _p(hh), 0, None, int(bool(is_w)), _p(out))
        return out
    idx = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.empty(idx.shape)
    _load().orc_heightfield_distance(nx, ny, nz, lx, ly, lz, _p(hh), int(idx.size),
                                     idx.ctypes.data_as(ctypes.c_void_p), int(bool(is_w)), _p(out))
    return out


def heightfield_sdf(grid, h2d, reach, nodes=None):
    """Sec. 3.1 with reading R10: phi = +d above the surface and -d below it, the
    side taken from z - h at the node's own column (a vertex of the surface), for
    every node within distance `reach` of the surface; beyond it phi = z - h
    (the same sign, and |z - h| >= d > reach).  Returns (phi_uv, phi_w): [nz, ny,
    nx] arrays, or the values at the flat indices `nodes` on each grid."""
    nx, ny, nz, lx, ly, lz = _shape(grid)
    dx, dy, dz = lx / nx, ly / ny, lz / (nz - 1)
    assert 0 < reach and reach + dx < 0.5 * lx and reach + dy < 0.5 * ly, "reach too large for the minimum image"
    hh = np.ascontiguousarray(h2d, dtype=np.float64)
    out = []
    for is_w in (False, True):
        if nodes is None:
            k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        else:
            flat = np.asarray(nodes, dtype=np.int64)
            i, j, k = flat % nx, (flat // nx) % ny, flat // (nx * ny)
        z = k * dz if is_w else (k + 0.5) * dz
        vertical = z - hh[j, i]
        d = heightfield_distance(grid, hh, is_w, nodes)
        out.append(np.where(d <= reach, np.sign(vertical) * d, vertical))
    return out[0], out[1]
