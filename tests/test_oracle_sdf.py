"""Pins of the oracle's height-field signed distance (Sec. 3.1: phi = +d in the
fluid, -d in the solid, d the minimum distance to the immersed boundary; the
surface through the sampled heights is piecewise linear, split along each cell's
(i, j)-(i+1, j+1) diagonal).  Each pin is fixed by something other than the
oracle's own formula: planes (closed-form distance |z - h| / sqrt(1 + |grad h|^2)),
a vertex apex, dense random sampling of the surface, the 1-Lipschitz property of
a distance, and convergence to the exact distance to the smooth ridge of Eq. 31
within the piecewise-linear interpolation bound."""
import numpy as np
import pytest

import oracle
from paper_2006_03343_gb300 import inputs


def _coords(grid, is_w):
    x, y, zu, zw = inputs.node_coords(grid)
    z = zw if is_w else zu
    return np.meshgrid(z, y, x, indexing="ij")[::-1]       # X, Y, Z as [nz, ny, nx]


def test_flat_surface_is_vertical_distance():
    grid = (12, 10, 9, 1.5, 1.0, 1.0)
    h = np.full((10, 12), 0.37)
    for reach in (0.05, 0.3):
        pu, pw = oracle.heightfield_sdf(grid, h, reach)
        for phi, is_w in ((pu, False), (pw, True)):
            _, _, z = _coords(grid, is_w)
            assert np.allclose(phi, z - 0.37, atol=1e-15, rtol=0)


def _tent_pin(grid, h, slope2, kink_dist, reach):
    """Nodes nearer to their own facet than to any kink line: d = |z - h| / sqrt(1 + slope2),
    slope2[ny, nx] the squared gradient of the facet under each column."""
    pu, pw = oracle.heightfield_sdf(grid, h, reach)
    du = oracle.heightfield_distance(grid, h, False)
    checked = 0
    for phi, d, is_w in ((pu, du, False), (pw, None, True)):
        x, y, z = _coords(grid, is_w)
        vert = z - h[None, :, :]
        plane = np.abs(vert) / np.sqrt(1.0 + slope2[None])
        sel = (plane < kink_dist(x, y)) & (plane <= reach * 0.999)
        assert sel.sum() > 20
        assert np.allclose(np.abs(phi[sel]), plane[sel], atol=1e-14, rtol=0)
        assert np.all(np.sign(phi[sel]) == np.sign(vert[sel]))
        checked += sel.sum()
    assert checked > 100


def test_tent_in_x_matches_plane_distance():
    nx, ny, nz = 32, 6, 24
    grid = (nx, ny, nz, 2.0, 1.0, 1.0)
    x = np.arange(nx) * (2.0 / nx)
    s, xc, hmax = 0.8, 1.0, 0.3
    h1 = np.maximum(0.0, hmax - s * np.abs(x - xc))            # kinks at x = 1, 0.625, 1.375 (all on columns)
    h = np.broadcast_to(h1[None, :], (ny, nx)).copy()
    kinks = np.array([xc, xc - hmax / s, xc + hmax / s, xc - 1.0 - hmax / s + 2.0, xc + 1.0 + hmax / s - 2.0])

    def kink_dist(X, Y):
        return np.min(np.abs(X[..., None] - kinks[None, None, None, :]), axis=-1)

    _tent_pin(grid, h, np.where(h > 0, s * s, 0.0), kink_dist, reach=0.2)


def test_tent_in_y_matches_plane_distance():
    nx, ny, nz = 6, 32, 24
    grid = (nx, ny, nz, 1.0, 2.0, 1.0)
    y = np.arange(ny) * (2.0 / ny)
    s, yc, hmax = 0.6, 0.75, 0.15
    h1 = np.maximum(0.0, hmax - s * np.abs(y - yc))            # kinks at 0.75, 0.5, 1.0
    h = np.broadcast_to(h1[:, None], (ny, nx)).copy()
    kinks = np.array([yc, yc - hmax / s, yc + hmax / s, yc + 2.0 - hmax / s, yc - 2.0 + hmax / s])

    def kink_dist(X, Y):
        return np.min(np.abs(Y[..., None] - kinks[None, None, None, :]), axis=-1)

    _tent_pin(grid, h, np.where(h > 0, s * s, 0.0), kink_dist, reach=0.2)


def test_diagonal_tent_pins_the_split_diagonal():
    """Kinks along lines i - j = const: the (i, j)-(i+1, j+1) split makes every
    triangle lie in one facet, so the plane distance |z - h| / sqrt(1 + 2 s^2)
    holds; the other diagonal would fold those cells."""
    n, nz = 24, 20
    L = 1.5
    grid = (n, n, nz, L, L, 1.0)
    d = L / n
    x = np.arange(n) * d
    s, hmax = 0.5, 0.125
    u = x[None, :] - x[:, None]                                  # x - y, [ny, nx]
    um = u - L * np.round(u / L)                                 # minimum image of x - y
    h = np.maximum(0.0, hmax - s * np.abs(um))                   # kinks at x - y = 0, +-0.25 (on node lines)
    assert np.allclose(hmax / s / d, round(hmax / s / d))

    def kink_dist(X, Y):
        w = X - Y
        w = w - L * np.round(w / L)
        ks = np.array([0.0, hmax / s, -hmax / s])
        gap = np.min(np.abs(w[..., None] - ks), axis=-1)
        return gap / np.sqrt(2.0)                                # distance to the kink line in the plane

    _tent_pin(grid, h, np.where(h > 0, 2 * s * s, 0.0), kink_dist, reach=0.15)


def test_apex_is_nearest_from_above():
    """The spike is the highest point of the surface, so for a node straight above it
    every other surface point s has (s - apex) . e_z <= 0 and lies no nearer."""
    grid = (20, 20, 16, 2.0, 2.0, 1.0)
    h = np.zeros((20, 20))
    h[12, 8] = 0.3
    pu, pw = oracle.heightfield_sdf(grid, h, 0.45)
    _, _, zw = _coords(grid, True)
    col = pw[:, 12, 8]
    above = zw[:, 12, 8] > 0.3
    assert above.sum() > 8
    assert np.allclose(col[above], zw[above, 12, 8] - 0.3, atol=1e-15)
    # far from the spike the surface is the floor: phi = z
    _, _, zu = _coords(grid, False)
    assert np.allclose(pu[:, 0, 0], zu[:, 0, 0], atol=1e-15)


def _sampled_distance(grid, h, p, per_tri, rng):
    """Minimum over random points of every surface triangle (and every periodic
    image shift in -1..1 of both directions) of the distance to p."""
    nx, ny, nz, lx, ly, lz = grid
    dx, dy = lx / nx, ly / ny
    best = np.inf
    a = rng.random((per_tri, 2))
    flip = a.sum(axis=1) > 1
    a[flip] = 1 - a[flip]                                       # uniform on the unit right triangle
    for j in range(ny):
        for i in range(nx):
            h00, h10 = h[j, i], h[j, (i + 1) % nx]
            h01, h11 = h[(j + 1) % ny, i], h[(j + 1) % ny, (i + 1) % nx]
            P00 = np.array([i * dx, j * dy, h00])
            P10 = np.array([(i + 1) * dx, j * dy, h10])
            P01 = np.array([i * dx, (j + 1) * dy, h01])
            P11 = np.array([(i + 1) * dx, (j + 1) * dy, h11])
            for A, B, C in ((P00, P10, P11), (P00, P11, P01)):
                pts = A + a[:, :1] * (B - A) + a[:, 1:] * (C - A)
                for sx in (-1, 0, 1):
                    for sy in (-1, 0, 1):
                        q = p - np.array([sx * lx, sy * ly, 0.0])
                        best = min(best, float(np.min(np.linalg.norm(pts - q, axis=1))))
    return best


def test_dense_surface_sampling_brackets_the_distance():
    rng = np.random.default_rng(7)
    grid = (5, 4, 8, 1.0, 0.8, 1.0)
    h = 0.2 + 0.25 * rng.random((4, 5))
    idx = rng.choice(5 * 4 * 8, size=12, replace=False)
    nx, ny, nz, lx, ly, lz = grid
    dx, dy, dz = lx / nx, ly / ny, lz / (nz - 1)
    for is_w in (False, True):
        d = oracle.heightfield_distance(grid, h, is_w, idx)
        for q, n in enumerate(idx):
            i, j, k = n % nx, (n // nx) % ny, n // (nx * ny)
            p = np.array([i * dx, j * dy, k * dz if is_w else (k + 0.5) * dz])
            ds = _sampled_distance(grid, h, p, 6000, rng)
            # samples lie on the surface, so they never beat the exact minimum; with
            # ~6000 points per triangle they come within a small fraction of a cell
            assert ds >= d[q] - 1e-12, (is_w, n, ds, d[q])
            assert ds <= d[q] + 0.02 * dx, (is_w, n, ds, d[q])


def test_distance_properties_on_random_terrain():
    """|d(p) - d(q)| <= |p - q| for neighbouring nodes (a distance is 1-Lipschitz),
    d <= |z - h| (the vertex below or above is on the surface), phi has the sign
    of z - h, and phi = z - h exactly where d exceeds the reach."""
    rng = np.random.default_rng(11)
    grid = (14, 12, 14, 1.4, 1.2, 1.0)
    nx, ny, nz, lx, ly, lz = grid
    h = inputs.gaussian_hills_height(grid, rng, nhills=3) + 0.05
    reach = 0.18
    pu, pw = oracle.heightfield_sdf(grid, h, reach)
    dx, dy, dz = lx / nx, ly / ny, lz / (nz - 1)
    for phi, is_w in ((pu, False), (pw, True)):
        d = oracle.heightfield_distance(grid, h, is_w)
        _, _, z = _coords(grid, is_w)
        vert = z - h[None]
        assert np.all(d <= np.abs(vert) + 1e-15)
        assert np.all(np.sign(phi) == np.sign(vert))
        far = d > reach
        assert far.any() and np.array_equal(phi[far], vert[far])
        assert np.allclose(np.abs(phi[~far]), d[~far], atol=0, rtol=0)
        for axis, step in ((2, dx), (1, dy), (0, dz)):
            diff = np.abs(np.diff(d, axis=axis)) if axis == 0 else np.abs(d - np.roll(d, 1, axis=axis))
            assert np.all(diff <= step + 1e-12), axis


def _ridge_exact_distance(px, pz, height, half_width, centre, period):
    """Distance from (px, pz) to the smooth cos^2 ridge of Eq. 31 (a curve in the
    x-z plane), by dense sampling around the node and a golden-section polish."""
    def h(x):
        r = x - centre
        r = r - period * np.round(r / period)
        return np.where(np.abs(r) < half_width, height * np.cos(np.pi * r / (2 * half_width)) ** 2, 0.0)

    xs = px + np.linspace(-0.5, 0.5, 200001)
    d2 = (xs - px) ** 2 + (h(xs) - pz) ** 2
    m = int(np.argmin(d2))
    a, b = xs[max(m - 1, 0)], xs[min(m + 1, xs.size - 1)]
    g = (np.sqrt(5) - 1) / 2
    f = lambda x: (x - px) ** 2 + (float(h(np.array(x))) - pz) ** 2
    for _ in range(80):
        c, e = b - g * (b - a), a + g * (b - a)
        if f(c) < f(e):
            b = e
        else:
            a = c
    return np.sqrt(f(0.5 * (a + b)))


@pytest.mark.parametrize("nx", [64, 128])
def test_converges_to_the_smooth_ridge(nx):
    """The piecewise-linear surface lies within max|h''| dx^2 / 8 of the smooth
    ridge, and the distance to two surfaces differs by at most their separation:
    |d_pl - d_exact| <= max|h''| dx^2 / 8 at every node near the ridge."""
    height, half_width, centre = 0.1, 0.3, 0.5
    grid = (nx, 4, 33, 1.0, 0.25, 1.0)
    hgt = inputs.ridge_height(grid, height=height, half_width=half_width, centre_frac=centre)
    dx = 1.0 / nx
    bound = height * (np.pi / (2 * half_width)) ** 2 * 2 * dx * dx / 8   # |h''| <= 2 H (pi / 2w)^2
    rng = np.random.default_rng(3)
    nodes = rng.choice(nx * 4 * 8, size=40, replace=False)          # the lowest 8 levels: near the ridge
    d = oracle.heightfield_distance(grid, hgt, True, nodes)
    dz = 1.0 / 32
    for q, n in enumerate(nodes):
        i, k = n % nx, n // (nx * 4)
        ex = _ridge_exact_distance(i * dx, k * dz, height, half_width, centre, 1.0)
        assert abs(d[q] - ex) <= bound + 1e-12, (n, d[q], ex, bound)


def test_reach_precondition():
    grid = (8, 8, 6, 1.0, 1.0, 1.0)
    with pytest.raises(AssertionError):
        oracle.heightfield_sdf(grid, np.zeros((8, 8)), 0.45)
