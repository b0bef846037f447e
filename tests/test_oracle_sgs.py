"""Pins of the oracle's Smagorinsky stress with Mason's wall damping (Eqs. 4-7):
the limits and the crossover of the damped mixing length; quadratic profiles
whose staggered differences are exact (they fix the placement of Eqs. 15-16 and
the level averages of |S|, including the floor rule); a horizontal sinusoid with
the known symbol sin(k d)/d of the central difference; the x <-> y mirror;
homogeneity of degree two; and the set of entries written (fluid nodes only,
the lid zeroed, floor and ghost levels kept).  None re-types the oracle: the
expected values are closed forms of the velocity fields, with lambda^2 from the
mixing length pinned on its own by the first test."""
import math

import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

CS, KAPPA = 0.16, 0.4


def _lam0(grid):
    nx, ny, nz, lx, ly, lz = grid
    return CS * (lx / nx * ly / ny * lz / (nz - 1)) ** (1.0 / 3.0)


def test_mixing_length_limits(oracle_mod):
    """Eq. 7, n = 2: lambda -> lambda_0 far from the wall, -> kappa (z + z0) close to
    it, lambda^2 = lambda_0^2 / 2 where the two are equal, and it grows with z."""
    grid = (16, 8, 9, 2.0, 1.0, 1.0)
    lam0 = _lam0(grid)
    z0 = 1e-4
    far = oracle_mod.mixing_length_sq(np.array([1e6]), z0, CS, KAPPA, grid)[0]
    assert far == pytest.approx(lam0 ** 2, rel=1e-9)
    near = oracle_mod.mixing_length_sq(np.array([1e-6]), z0, CS, KAPPA, grid)[0]
    assert near == pytest.approx((KAPPA * (1e-6 + z0)) ** 2, rel=1e-4)
    cross = lam0 / KAPPA - z0
    assert oracle_mod.mixing_length_sq(np.array([cross]), z0, CS, KAPPA, grid)[0] == pytest.approx(
        lam0 ** 2 / 2, rel=1e-12)
    zs = np.linspace(0.0, 1.0, 50)
    lam = oracle_mod.mixing_length_sq(zs, z0, CS, KAPPA, grid)
    assert np.all(np.diff(lam) > 0) and np.all(lam < lam0 ** 2)


def _all_fluid(shape, lengths=(2.0, 1.0, 1.0), depth=0.5):
    """A flat wall `depth` below the floor: every node is fluid (phi > 2 phi_b)."""
    nx, ny, nz = shape
    grid = (nx, ny, nz) + tuple(lengths)
    x, y, z_uv, z_w = inputs.node_coords(grid)
    phi_uv = np.ascontiguousarray(np.broadcast_to((z_uv + depth)[:, None, None], (nz, ny, nx)))
    phi_w = np.ascontiguousarray(np.broadcast_to((z_w + depth)[:, None, None], (nz, ny, nx)))
    return grid, x, y, z_uv, z_w, phi_uv, phi_w


def _run(oracle_mod, grid, phi_uv, phi_w, u, v, w, z0=1e-4, phi_b=None, fill=7.0):
    nz = grid[2]
    phi_b = 0.5 * grid[5] / (nz - 1) if phi_b is None else phi_b
    tau = {k: np.full(u.shape, fill) for k in inputs.TAU_NAMES}
    oracle_mod.sgs_stress(grid, phi_uv, phi_w, z0, phi_b, u, v, w, tau, cs=CS, kappa=KAPPA)
    return tau


def test_quadratic_shear_places_the_vertical_differences(oracle_mod):
    """u = a z^2 + c sin(k x) on uv-levels, v = w = 0.  S11 = c sin(k dx)/dx cos(k x)
    on every uv-node.  On w-node k the difference of Eq. 15 is exactly 2 a z_w, so
    S13 = a z_w and |S|^2 = 2 S11^2 + 4 S13^2 there.  On uv-node k,
    |S|^2 = 2 S11^2 + 4 s^2 with s the mean S13 of the w-levels around it: a z_uv,
    except on level 0 where the floor repeats level 1 (s = a dz) and on the top
    level, whose upper neighbour is the stress-free lid (s = a z_w / 2)."""
    nx, ny, nz = 16, 4, 9
    grid, x, y, z_uv, z_w, phi_uv, phi_w = _all_fluid((nx, ny, nz))
    dx, dz = grid[3] / nx, grid[5] / (nz - 1)
    a, c, k = 1.7, 0.3, 2 * math.pi * 3 / grid[3]
    shp = (nz, ny, nx)
    u = np.ascontiguousarray(np.broadcast_to(a * z_uv[:, None, None] ** 2 + c * np.sin(k * x)[None, None, :], shp))
    zero = np.zeros(shp)
    tau = _run(oracle_mod, grid, phi_uv, phi_w, u, zero, zero)
    lam_w = oracle_mod.mixing_length_sq(phi_w, 1e-4, CS, KAPPA, grid)
    lam_uv = oracle_mod.mixing_length_sq(phi_uv, 1e-4, CS, KAPPA, grid)
    s11 = c * math.sin(k * dx) / dx * np.cos(k * x)[None, None, :]
    s13 = a * z_w[1:-1, None, None]
    # on a w-node the mean S11 of the uv-levels around it is S11 itself (it does not vary with z)
    exp_xz = -2.0 * lam_w[1:-1] * np.sqrt(2 * s11 ** 2 + 4 * s13 ** 2) * s13
    np.testing.assert_allclose(tau["txz"][1:-1], np.broadcast_to(exp_xz, (nz - 2, ny, nx)), rtol=1e-12, atol=1e-15)
    s = a * z_uv[:-1, None, None] * np.ones((nz - 1, 1, 1))
    s[0] = a * dz                          # the floor repeats w-level 1
    s[-1] = 0.5 * a * z_w[nz - 2]          # the lid carries no strain (no stress there, Eq. 10)
    mag = np.sqrt(2 * s11 ** 2 + 4 * s ** 2)
    np.testing.assert_allclose(tau["txx"][:-1], -2.0 * lam_uv[:-1] * mag * s11, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(tau["tyy"][:-1], 0.0, atol=1e-15)
    np.testing.assert_allclose(tau["tyz"][1:-1], 0.0, atol=1e-15)


def test_quadratic_w_places_the_uv_difference(oracle_mod):
    """w = b z^2 on w-levels: Eq. 16 gives S33 = 2 b z_uv exactly on uv-node k, so
    tau_zz = -2 sqrt(2) lambda^2 |S33| S33; S13 = S23 = 0."""
    nx, ny, nz = 8, 6, 11
    grid, x, y, z_uv, z_w, phi_uv, phi_w = _all_fluid((nx, ny, nz))
    b = -0.9
    shp = (nz, ny, nx)
    w = np.ascontiguousarray(np.broadcast_to(b * z_w[:, None, None] ** 2, shp))
    zero = np.zeros(shp)
    tau = _run(oracle_mod, grid, phi_uv, phi_w, zero, zero, w)
    lam_uv = oracle_mod.mixing_length_sq(phi_uv, 1e-4, CS, KAPPA, grid)
    s33 = 2 * b * z_uv[:-1, None, None]
    np.testing.assert_allclose(tau["tzz"][:-1], -2.0 * math.sqrt(2.0) * lam_uv[:-1] * np.abs(s33) * s33, rtol=1e-12)
    np.testing.assert_allclose(tau["txz"][1:-1], 0.0, atol=1e-15)


def test_horizontal_sinusoid_symbol(oracle_mod):
    """u = A sin(k y): S12 = A/2 sin(k dy)/dy cos(k y) and |S| = 2 |S12|, so
    tau_xy = -4 lambda^2 |S12| S12 on every fluid uv-node."""
    nx, ny, nz = 6, 24, 5
    grid, x, y, z_uv, z_w, phi_uv, phi_w = _all_fluid((nx, ny, nz), lengths=(1.0, 3.0, 1.0))
    dy = grid[4] / ny
    A, k = 2.5, 2 * math.pi * 5 / grid[4]
    shp = (nz, ny, nx)
    u = np.ascontiguousarray(np.broadcast_to(A * np.sin(k * y)[None, :, None], shp))
    zero = np.zeros(shp)
    tau = _run(oracle_mod, grid, phi_uv, phi_w, u, zero, zero)
    lam_uv = oracle_mod.mixing_length_sq(phi_uv, 1e-4, CS, KAPPA, grid)
    s12 = 0.5 * A * math.sin(k * dy) / dy * np.cos(k * y)[None, :, None]
    np.testing.assert_allclose(tau["txy"][:-1], -4.0 * lam_uv[:-1] * np.abs(s12) * s12, rtol=1e-12, atol=1e-15)


def test_mirror_x_y(oracle_mod):
    """On a square-celled grid, swapping x and y (transposing the fields, exchanging
    u and v) exchanges txx with tyy and txz with tyz and transposes txy, tzz."""
    n, nz = 12, 7
    grid = (n, n, nz, 1.0, 1.0, 1.0)
    rng = np.random.default_rng(3)
    shp = (nz, n, n)
    u, v, w = (rng.standard_normal(shp) for _ in range(3))
    _, x, y, z_uv, z_w, phi_uv, phi_w = _all_fluid((n, n, nz), lengths=(1.0, 1.0, 1.0))
    t1 = _run(oracle_mod, grid, phi_uv, phi_w, u, v, w)
    T = lambda a: np.ascontiguousarray(np.swapaxes(a, 1, 2))
    t2 = _run(oracle_mod, grid, phi_uv, phi_w, T(v), T(u), T(w))
    for a, b in (("txx", "tyy"), ("tyy", "txx"), ("txz", "tyz"), ("tyz", "txz"), ("txy", "txy"), ("tzz", "tzz")):
        np.testing.assert_allclose(T(t2[b]), t1[a], rtol=1e-12, atol=1e-14)


def test_homogeneity_and_dissipation(oracle_mod):
    """tau(alpha u) = alpha |alpha| tau(u); and on uv-nodes the products with the
    strain of the same node sum to <= 0 (nu_t >= 0)."""
    grid, x, y, z_uv, z_w, phi_uv, phi_w = _all_fluid((10, 8, 6))
    rng = np.random.default_rng(5)
    shp = (6, 8, 10)
    u, v, w = (rng.standard_normal(shp) for _ in range(3))
    t1 = _run(oracle_mod, grid, phi_uv, phi_w, u, v, w)
    alpha = -1.7
    t2 = _run(oracle_mod, grid, phi_uv, phi_w, alpha * u, alpha * v, alpha * w)
    for k in inputs.TAU_NAMES:
        inner = (slice(None, -1) if k in ("txx", "tyy", "tzz", "txy") else slice(1, -1))
        np.testing.assert_allclose(t2[k][inner], alpha * abs(alpha) * t1[k][inner], rtol=1e-12, atol=1e-14)
    dx, dy, dz = 2.0 / 10, 1.0 / 8, 1.0 / 5
    s11 = (np.roll(u, -1, 2) - np.roll(u, 1, 2)) / (2 * dx)
    s22 = (np.roll(v, -1, 1) - np.roll(v, 1, 1)) / (2 * dy)
    s12 = 0.5 * ((np.roll(u, -1, 1) - np.roll(u, 1, 1)) / (2 * dy) + (np.roll(v, -1, 2) - np.roll(v, 1, 2)) / (2 * dx))
    s33 = (w[1:] - w[:-1]) / dz
    prod = (t1["txx"][:-1] * s11[:-1] + t1["tyy"][:-1] * s22[:-1] + t1["tzz"][:-1] * s33
            + 2 * t1["txy"][:-1] * s12[:-1])
    assert np.all(prod <= 1e-14)


def test_entries_written(oracle_mod):
    """On the ridge terrain: fluid entries change, band and solid entries, the ghost
    uv-level and the floor w-level keep their values, the lid's fluid tau_xz, tau_yz
    are 0."""
    case = inputs.ridge(shape=(24, 16, 12))
    fill = 7.0
    tau = {k: np.full(case.u.shape, fill) for k in inputs.TAU_NAMES}
    oracle_mod.sgs_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_b, case.u, case.v, case.w, tau)
    cu, cw = oracle_mod.classify(case.grid, case.phi_uv, case.phi_w, case.phi_b)
    for k in ("txx", "tyy", "tzz", "txy"):
        t = tau[k]
        assert np.all(t[-1] == fill)
        assert np.all(t[:-1][cu[:-1] != 0] == fill)
        assert np.all(t[:-1][cu[:-1] == 0] != fill)
    for k in ("txz", "tyz"):
        t = tau[k]
        assert np.all(t[0] == fill)
        assert np.all(t[-1][cw[-1] == 0] == 0.0) and np.all(t[-1][cw[-1] != 0] == fill)
        assert np.all(t[1:-1][cw[1:-1] != 0] == fill)
        assert np.all(t[1:-1][cw[1:-1] == 0] != fill)
