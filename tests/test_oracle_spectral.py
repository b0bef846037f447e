"""Pins of the oracle's pseudo-spectral divergence (Eqs. 13-14 for the horizontal
derivatives, Eqs. 15-16 for the vertical ones, f = -div tau of Eq. 2 / Eq. 18).

None of these re-types the oracle: single Fourier modes have closed-form
derivatives; the Nyquist mode and the mean carry none; a direct O(N^2) evaluation
of the Fourier sums (no FFT) on a tiny grid; skew-adjointness of d/dx; the known
symbols of the central difference (sin(k dx)/dx) and of the spectral derivative
(k); and the telescoping of periodic plane sums.
"""
import math

import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs


def _coords(grid):
    x, y, z_uv, z_w = inputs.node_coords(grid)
    return x[None, None, :], y[None, :, None], z_uv[:, None, None], z_w[:, None, None]


@pytest.mark.parametrize("shape,lengths", [((16, 8, 6), (2 * math.pi, math.pi, 1.0)),
                                           ((12, 10, 5), (3.0, 1.7, 0.8)),
                                           ((32, 32, 4), (1.0, 1.0, 1.0))])
def test_single_modes_have_closed_form_derivatives(oracle_mod, shape, lengths):
    """Eqs. 13-14 differentiate every resolved mode exactly: with each stress a single
    mode (wavenumber below Nyquist) times a function of z, plus terms linear in z for
    the vertical parts, f equals the analytic -div tau to rounding."""
    nx, ny, nz = shape
    grid = shape + lengths
    X, Y, Zuv, Zw = _coords(grid)
    kx = lambda m: 2 * math.pi * m / lengths[0]
    ky = lambda m: 2 * math.pi * m / lengths[1]
    s = 1.0 + 0.5 * Zuv                               # arbitrary level dependence on uv-levels
    a = dict(txx=(3, 1, 0.3), txy=(-2, 2, -0.7), tyy=(1, -3, 1.1), txz=(nx // 2 - 1, 1, 0.2),
             tyz=(2, -(ny // 2 - 1), 0.9), tzz=(-1, 1, -0.4))
    c1, c2, c3 = 0.75, -1.25, 2.5
    ph = {k: kx(m) * X + ky(n) * Y + p for k, (m, n, p) in a.items()}
    zero = 0 * X * Y * Zw
    tau = dict(txx=s * np.cos(ph["txx"]), txy=s * np.sin(ph["txy"]), tyy=s * np.cos(ph["tyy"]),
               txz=c1 * Zw + np.cos(ph["txz"]) + zero, tyz=c2 * Zw + np.sin(ph["tyz"]) + zero,
               tzz=c3 * Zuv + np.cos(ph["tzz"]) + zero)
    tau = {k: np.ascontiguousarray(np.broadcast_to(v, (nz, ny, nx))) for k, v in tau.items()}
    d_txx_dx = -s * kx(a["txx"][0]) * np.sin(ph["txx"])
    d_txy_dy = s * ky(a["txy"][1]) * np.cos(ph["txy"])
    d_txy_dx = s * kx(a["txy"][0]) * np.cos(ph["txy"])
    d_tyy_dy = -s * ky(a["tyy"][1]) * np.sin(ph["tyy"])
    d_txz_dx = -kx(a["txz"][0]) * np.sin(ph["txz"])
    d_tyz_dy = ky(a["tyz"][1]) * np.cos(ph["tyz"])
    fx_ref = np.broadcast_to(-(d_txx_dx + d_txy_dy + c1), (nz, ny, nx)).copy()
    fy_ref = np.broadcast_to(-(d_txy_dx + d_tyy_dy + c2), (nz, ny, nx)).copy()
    fz_ref = np.broadcast_to(-(d_txz_dx + d_tyz_dy + c3), (nz, ny, nx)).copy()
    fx_ref[-1] = fy_ref[-1] = 0.0                     # ghost uv-level
    fz_ref[0] = fz_ref[-1] = 0.0                      # floor and lid
    fx, fy, fz = oracle_mod.force_spectral(grid, tau)
    for got, ref in ((fx, fx_ref), (fy, fy_ref), (fz, fz_ref)):
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-12 * scale
    assert np.all(fx[-1] == 0) and np.all(fy[-1] == 0) and np.all(fz[0] == 0) and np.all(fz[-1] == 0)


def test_nyquist_and_mean_carry_no_derivative(oracle_mod):
    """(-1)^i, (-1)^j and constants have zero horizontal derivative (the Nyquist mode
    is not differentiated, the mean has k = 0)."""
    nx, ny, nz = 8, 6, 4
    grid = (nx, ny, nz, 2.0, 1.0, 1.0)
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    a = np.ascontiguousarray(np.broadcast_to((-1.0) ** i + 2.0 * (-1.0) ** j + 3.0, (nz, ny, nx)))
    ddx, ddy = oracle_mod.horizontal_derivatives(grid, a)
    assert np.abs(ddx).max() <= 1e-13 and np.abs(ddy).max() <= 1e-13


def _direct_sums(grid, a):
    """Eqs. 13-14 evaluated literally: the Fourier amplitude of each resolved
    (k_x, k_y) by a direct sum over the plane, then the synthesis sum with i k_x and
    i k_y.  Resolved integer modes m run over -n/2 < m <= n/2; the highest one of an
    even n is the Nyquist mode, whose derivative is taken as zero."""
    nx, ny, nz, lx, ly, lz = grid
    x = np.arange(nx) * lx / nx
    y = np.arange(ny) * ly / ny
    mxs = [m for m in range(-(nx // 2), nx // 2 + 1) if -nx / 2 < m <= nx / 2]
    mys = [m for m in range(-(ny // 2), ny // 2 + 1) if -ny / 2 < m <= ny / 2]
    ddx = np.zeros(a.shape)
    ddy = np.zeros(a.shape)
    for k in range(nz):
        for mx in mxs:
            kx = 2 * math.pi * mx / lx
            for my in mys:
                ky = 2 * math.pi * my / ly
                amp = 0j
                for jj in range(ny):
                    for ii in range(nx):
                        amp += a[k, jj, ii] * complex(math.cos(kx * x[ii] + ky * y[jj]),
                                                      -math.sin(kx * x[ii] + ky * y[jj]))
                amp /= nx * ny
                dkx = 0.0 if (nx % 2 == 0 and mx == nx // 2) else kx
                dky = 0.0 if (ny % 2 == 0 and my == ny // 2) else ky
                for jj in range(ny):
                    for ii in range(nx):
                        e = complex(math.cos(kx * x[ii] + ky * y[jj]), math.sin(kx * x[ii] + ky * y[jj]))
                        ddx[k, jj, ii] += (1j * dkx * amp * e).real
                        ddy[k, jj, ii] += (1j * dky * amp * e).real
    return ddx, ddy


@pytest.mark.parametrize("shape", [(8, 4, 2), (6, 5, 2), (4, 8, 1)])
def test_direct_fourier_sums(oracle_mod, shape):
    """Brute force on tiny grids (even and odd sizes): the FFT-based derivatives equal
    the literal double sums of Eqs. 13-14."""
    nx, ny, nz = shape
    grid = (nx, ny, nz, 1.3, 0.9, 1.0)
    a = np.random.default_rng(3).standard_normal((nz, ny, nx))
    ddx, ddy = oracle_mod.horizontal_derivatives(grid, a)
    rx, ry = _direct_sums(grid, a)
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    assert np.abs(ddx - rx).max() <= 1e-12 * scale
    assert np.abs(ddy - ry).max() <= 1e-12 * scale


def test_derivatives_are_skew_adjoint(oracle_mod):
    """<g, d/dx q> = -<d/dx g, q> (and the same for y) for random periodic fields."""
    rng = np.random.default_rng(8)
    grid = (16, 12, 3, 2.0, 1.5, 1.0)
    g = rng.standard_normal((3, 12, 16))
    q = rng.standard_normal((3, 12, 16))
    gx, gy = oracle_mod.horizontal_derivatives(grid, g)
    qx, qy = oracle_mod.horizontal_derivatives(grid, q)
    assert abs(np.sum(g * qx) + np.sum(gx * q)) <= 1e-11 * np.sum(np.abs(g * qx))
    assert abs(np.sum(g * qy) + np.sum(gy * q)) <= 1e-11 * np.sum(np.abs(g * qy))


@pytest.mark.parametrize("m", [1, 5, 13])
def test_symbols_of_central_and_spectral_derivatives(oracle_mod, m):
    """For txx = sin(k x) the central-difference divergence gives -sin(k dx)/dx cos(k x)
    and the spectral one -k cos(k x): the two forms differ exactly by their symbols."""
    nx, ny, nz = 32, 4, 3
    lx = 2.0
    grid = (nx, ny, nz, lx, 1.0, 1.0)
    dx = lx / nx
    k = 2 * math.pi * m / lx
    X = (np.arange(nx) * dx)[None, None, :]
    tau = {n: np.zeros((nz, ny, nx)) for n in inputs.TAU_NAMES}
    tau["txx"] = np.ascontiguousarray(np.broadcast_to(np.sin(k * X), (nz, ny, nx)))
    fd = oracle_mod.force(grid, tau)[0]
    sp = oracle_mod.force_spectral(grid, tau)[0]
    c = np.broadcast_to(np.cos(k * X), (nz, ny, nx))[:-1]
    assert np.abs(fd[:-1] + math.sin(k * dx) / dx * c).max() <= 1e-12 * k
    assert np.abs(sp[:-1] + k * c).max() <= 1e-12 * k


def test_plane_sums_telescope(oracle_mod):
    """Horizontal derivatives of periodic fields sum to zero over a plane, so
    sum_ij f_x = -sum_ij (txz[k+1] - txz[k]) / dz level by level (and likewise f_y, f_z)."""
    rng = np.random.default_rng(21)
    nx, ny, nz = 16, 8, 7
    grid = (nx, ny, nz, 1.0, 0.5, 1.0)
    dz = 1.0 / (nz - 1)
    tau = {n: rng.standard_normal((nz, ny, nx)) for n in inputs.TAU_NAMES}
    fx, fy, fz = oracle_mod.force_spectral(grid, tau)
    sxz = tau["txz"].sum(axis=(1, 2))
    syz = tau["tyz"].sum(axis=(1, 2))
    szz = tau["tzz"].sum(axis=(1, 2))
    np.testing.assert_allclose(fx.sum(axis=(1, 2))[:-1], -(sxz[1:] - sxz[:-1]) / dz, rtol=0, atol=1e-10)
    np.testing.assert_allclose(fy.sum(axis=(1, 2))[:-1], -(syz[1:] - syz[:-1]) / dz, rtol=0, atol=1e-10)
    np.testing.assert_allclose(fz.sum(axis=(1, 2))[1:-1], -(szz[1:-1] - szz[:-2]) / dz, rtol=0, atol=1e-10)
