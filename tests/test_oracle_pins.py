"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it rests on.  None of them re-types an oracle
formula: they use closed forms (the flat-wall log law of Eqs. 9-10 and 29),
hand-derived node classes (the raised flat walls of Sec. 4.1), brute force
(tent-function interpolation), algebraic identities of the rotation
tau_ij = a_im a_jn tau'_mn, exact derivatives of polynomials and sinusoids for
the divergence, and set identities for the body mask (Eq. 27).
"""
import math

import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

KAPPA = 0.4


def _fresh_tau(shape, fill=np.nan):
    return {k: np.full(shape, fill) for k in inputs.TAU_NAMES}


# --------------------------------------------------------------------------- #
# T1: flat terrain phi = z with a pure log profile reproduces tau_w = -u*^2
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("theta", [0.0, 0.7, -2.1])
@pytest.mark.parametrize("field_z0", [False, True])
def test_flat_wall_log_law(oracle_mod, theta, field_z0):
    """Sec. 2.3 Eqs. 9-10 and Sec. 4.1 Eq. 29: with u = (u*/kappa) ln(z/z0) along a
    horizontal direction theta and the sample point on a uv-node (phi_c = 1.5 dz),
    the w-band stress is tau_xz = -u*^2 cos(theta), tau_yz = -u*^2 sin(theta) and the
    uv-band stresses vanish (n has no horizontal part, U_r no vertical part)."""
    nx, ny, nz = 8, 6, 33                     # dz = 1/32 exactly
    grid = (nx, ny, nz, 1.0, 1.0, 1.0)
    dz = 1.0 / 32
    z0, ustar = 1e-4, 1.3
    z_uv = (np.arange(nz) + 0.5) * dz
    z_w = np.arange(nz) * dz
    phi_uv = np.ascontiguousarray(np.broadcast_to(z_uv[:, None, None], (nz, ny, nx)))
    phi_w = np.ascontiguousarray(np.broadcast_to(z_w[:, None, None], (nz, ny, nx)))
    prof = (ustar / KAPPA) * np.log(z_uv / z0)
    u = np.ascontiguousarray(np.broadcast_to((prof * math.cos(theta))[:, None, None], (nz, ny, nx)))
    v = np.ascontiguousarray(np.broadcast_to((prof * math.sin(theta))[:, None, None], (nz, ny, nx)))
    w = np.zeros((nz, ny, nx))
    tau = _fresh_tau((nz, ny, nx), 7.0)
    z0_arg = np.full((nz, ny, nx), z0) if field_z0 else z0
    stats = oracle_mod.wall_stress(grid, phi_uv, phi_w, z0_arg, 1.5 * dz, 0.5 * dz, u, v, w, tau)

    np.testing.assert_allclose(tau["txz"][0], -ustar ** 2 * math.cos(theta), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(tau["tyz"][0], -ustar ** 2 * math.sin(theta), rtol=1e-13, atol=1e-13)
    for name in ("txx", "txy", "tyy", "tzz"):
        np.testing.assert_allclose(tau[name][0], 0.0, atol=1e-13)
    # every other node is fluid: its stress passes through untouched
    for name in inputs.TAU_NAMES:
        assert np.all(tau[name][1:] == 7.0)
    # stats: one band layer per grid, tau_w = -u*^2 everywhere on the w-band
    assert stats[0, 0] == nx * ny and stats[1, 0] == nx * ny
    np.testing.assert_allclose(stats[0, 1], -nx * ny * ustar ** 2, rtol=1e-13)
    np.testing.assert_allclose(stats[0, 2], nx * ny * ustar ** 4, rtol=1e-13)
    np.testing.assert_allclose(stats[0, 3], -ustar ** 2, rtol=1e-13)
    np.testing.assert_allclose(stats[0, 4], (ustar / KAPPA) * math.log(1.5 * dz / z0), rtol=1e-13)
    assert stats[0, 5] == 0 and stats[1, 5] == 0          # x_c = 1.5 dz lies inside both grids


# --------------------------------------------------------------------------- #
# reading R3: sample points beyond the physical levels are clamped, and counted
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("above", [False, True])
def test_zclamp_count_flat_wall_near_lid(oracle_mod, above):
    """A flat wall at height h (phi = z - h, n = (0,0,1) exactly): every band node
    samples at z_c = h + phi_c (Sec. 3.3, reading R2).  The top physical uv-level is
    (nz - 1.5) dz (the level nz - 1 lies above the lid) and the top w-level (nz - 1) dz,
    so the interpolation clamps every band node's sample point exactly when
    h + phi_c > (nz - 1.5) dz, and none otherwise.  The clamped sample takes the top
    uv-level's velocity; w is 0 there in this field."""
    nx, ny, nz = 8, 6, 17
    dz = 1.0 / (nz - 1)
    phi_c = 1.5 * dz
    top_uv = (nz - 1.5) * dz
    h = top_uv - phi_c + (0.2 if above else -0.2) * dz
    grid = (nx, ny, nz, 1.0, 1.0, 1.0)
    z_uv = (np.arange(nz) + 0.5) * dz
    z_w = np.arange(nz) * dz
    phi_uv = np.ascontiguousarray(np.broadcast_to((z_uv - h)[:, None, None], (nz, ny, nx)))
    phi_w = np.ascontiguousarray(np.broadcast_to((z_w - h)[:, None, None], (nz, ny, nx)))
    rng = np.random.default_rng(11)
    u = rng.standard_normal((nz, ny, nx))
    v = rng.standard_normal((nz, ny, nx))
    w = rng.standard_normal((nz, ny, nx))
    tau = _fresh_tau((nz, ny, nx), 0.0)
    stats = oracle_mod.wall_stress(grid, phi_uv, phi_w, 1e-4, phi_c, 0.5 * dz, u, v, w, tau)
    assert stats[0, 0] > 0 and stats[1, 0] > 0
    for b in range(2):
        assert stats[b, 5] == (stats[b, 0] if above else 0)


# --------------------------------------------------------------------------- #
# T2: node classes of the raised flat walls of Sec. 4.1 (cases 1-4)
# --------------------------------------------------------------------------- #
# levels derived by hand from the inequalities of Sec. 3.3 with phi_b = dz/2:
#   w-node k at z = k dz, phi = (k - c) dz, band |k - c| <= 1/2, solid k - c < -1/2
#   uv-node k at z = (k + 1/2) dz, phi = (k + 1/2 - c) dz, band 0 <= . <= 1, solid < 0
RAISED = {
    1.0: dict(w_band={1}, w_solid={0}, uv_band={1}, uv_solid={0}),
    1.25: dict(w_band={1}, w_solid={0}, uv_band={1}, uv_solid={0}),
    1.5: dict(w_band={1, 2}, w_solid={0}, uv_band={1, 2}, uv_solid={0}),
    1.75: dict(w_band={2}, w_solid={0, 1}, uv_band={2}, uv_solid={0, 1}),
}


@pytest.mark.parametrize("c", sorted(RAISED))
def test_raised_flat_wall_classes(oracle_mod, c):
    """Sec. 3.3 classes on the paper's 64 x 32 x 33 flat-terrain grid (Sec. 4.1),
    wall at z_w/dz = c; the tie case c = 1.5 puts two levels in each band."""
    case = inputs.flat((64, 32, 33), wall_height=c / 32.0, lengths=(8.0, 4.0, 1.0))
    cu, cw = oracle_mod.classify(case.grid, case.phi_uv, case.phi_w, case.phi_b)
    exp = RAISED[c]
    for cls, grid_name in ((cw, "w"), (cu, "uv")):
        band = {int(k) for k in np.unique(np.nonzero(cls == 1)[0])}
        solid = {int(k) for k in np.unique(np.nonzero(cls == 2)[0])}
        assert band == exp[f"{grid_name}_band"]
        assert solid == exp[f"{grid_name}_solid"]
        # classes are per level: every column identical
        for k in range(case.grid[2]):
            assert np.all(cls[k] == cls[k, 0, 0])


@pytest.mark.parametrize("c,first_is_w", [(1.0, False), (1.25, False), (1.5, True), (1.75, True)])
def test_first_node_above_wall(c, first_is_w):
    """Sec. 4.1: for cases 3 and 4 the first node above the surface is a w-node,
    for cases 1 and 2 a uv-node.  Pins the vertical staggering (Sec. 2.4)."""
    case = inputs.flat((4, 4, 33), wall_height=c / 32.0)
    first_uv = np.min(np.where(case.phi_uv[:, 0, 0] > 0, np.arange(33) + 0.5, np.inf))
    first_w = np.min(np.where(case.phi_w[:, 0, 0] > 0, np.arange(33) + 0.0, np.inf))
    assert (first_w < first_uv) == first_is_w


# --------------------------------------------------------------------------- #
# T3: tilted plane, uniform velocity: closed form and rotation covariance
# --------------------------------------------------------------------------- #
def _plane_case(normal, offset, uvec, shape=(24, 20, 25), lengths=(1.2, 1.0, 1.0)):
    nx, ny, nz = shape
    grid = (nx, ny, nz) + tuple(lengths)
    x, y, z_uv, z_w = inputs.node_coords(grid)
    nrm = np.asarray(normal, float) / np.linalg.norm(normal)
    X = x[None, None, :]
    Y = y[None, :, None]
    phi_uv = np.ascontiguousarray(nrm[0] * X + nrm[1] * Y + nrm[2] * z_uv[:, None, None] - offset + 0 * X * Y)
    phi_w = np.ascontiguousarray(nrm[0] * X + nrm[1] * Y + nrm[2] * z_w[:, None, None] - offset + 0 * X * Y)
    u = np.full((nz, ny, nx), float(uvec[0]))
    v = np.full((nz, ny, nx), float(uvec[1]))
    w = np.full((nz, ny, nx), float(uvec[2]))
    return grid, phi_uv, phi_w, u, v, w, nrm


def _closed_form(nrm, uvec, C):
    uvec = np.asarray(uvec, float)
    Ur = uvec - np.dot(uvec, nrm) * nrm
    mag = np.linalg.norm(Ur)
    return -C * mag * (np.outer(Ur, nrm) + np.outer(nrm, Ur)), -C * mag * mag, mag


@pytest.mark.parametrize("normal,uvec", [
    ((0.3, 0.0, 1.0), (2.0, 0.5, 0.1)),
    ((-0.2, 0.25, 1.0), (1.5, -0.7, 0.3)),
    ((0.0, -0.4, 1.0), (0.2, 3.0, -0.2)),
])
def test_tilted_plane_closed_form(oracle_mod, normal, uvec):
    """Sec. 3.3: for a plane phi = n.x - d the central differences give n exactly and
    the interpolation of a uniform velocity is exact, so tau must equal the rotated
    local tensor with tau'_13 = tau'_31 = tau_w, which by hand is
    tau = tau_w (t n^T + n t^T), t = U_r/|U_r|, tau_w = -[kappa U_r / ln(phi_c/z0)]^2."""
    z0, phi_c = 1e-3, 0.06
    grid, phi_uv, phi_w, u, v, w, nrm = _plane_case(normal, 0.3, uvec)
    nx, ny, nz = grid[:3]
    C = (KAPPA / math.log(phi_c / z0)) ** 2
    tref, twref, urref = _closed_form(nrm, uvec, C)
    checked = 0
    for is_w, phi in ((1, phi_w), (0, phi_uv)):
        for k in range(1, nz - 2):
            for j in range(0, ny, 3):
                for i in range(1, nx - 1):        # keep the x stencil off the periodic seam
                    if abs(phi[k, j, i]) > 0.05:
                        continue
                    if j in (0, ny - 1) and nrm[1] != 0:
                        continue
                    t, tw, ur = oracle_mod.wall_model_node(grid, phi, is_w, i, j, k, u, v, w, z0, phi_c)
                    np.testing.assert_allclose(t, tref, rtol=1e-12, atol=1e-12)
                    assert t[0, 2] == pytest.approx(t[2, 0], rel=1e-14, abs=1e-15)
                    np.testing.assert_allclose(tw, twref, rtol=1e-12)
                    np.testing.assert_allclose(ur, urref, rtol=1e-12)
                    checked += 1
    assert checked > 20


def test_rotation_covariance(oracle_mod):
    """tau_ij = a_im a_jn tau'_mn is a tensor: turning the whole configuration by
    90 degrees about z (x -> y, y -> -x) turns tau into R tau R^T."""
    z0, phi_c = 1e-3, 0.06
    n1, u1 = np.array([0.3, 0.1, 1.0]), np.array([1.7, 0.4, 0.2])
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    n2, u2 = R @ n1, R @ u1
    g1 = _plane_case(n1, 0.3, u1, shape=(20, 20, 25), lengths=(1.0, 1.0, 1.0))
    # configuration 2 is configuration 1 turned about z and shifted by one period
    # in x (x2 = L - y1), so that its nodes are the images of configuration 1's
    g2 = _plane_case(n2, 0.3 + (n2 / np.linalg.norm(n2))[0] * 1.0, u2, shape=(20, 20, 25),
                     lengths=(1.0, 1.0, 1.0))
    k, j, i = 9, 8, 10
    grid1, phi1 = g1[0], g1[2]
    # pick a band node of configuration 1 and its image in configuration 2
    k = int(np.argmin(np.abs(phi1[:, j, i])))
    t1, tw1, _ = oracle_mod.wall_model_node(grid1, g1[2], 1, i, j, k, *g1[3:6], z0, phi_c)
    # (i, j) -> rotated node: x2 = -y1, y2 = x1 on the same square lattice
    i2, j2 = (-j) % 20, i
    t2, tw2, _ = oracle_mod.wall_model_node(g2[0], g2[2], 1, i2, j2, k, *g2[3:6], z0, phi_c)
    assert g2[2][k, j2, i2] == pytest.approx(phi1[k, j, i], abs=1e-12)
    np.testing.assert_allclose(t2, R @ t1 @ R.T, rtol=1e-12, atol=1e-13)
    assert tw2 == pytest.approx(tw1, rel=1e-12)


# --------------------------------------------------------------------------- #
# T4: interpolation equals brute-force periodic tent weights
# --------------------------------------------------------------------------- #
def test_interp_brute_force(oracle_mod):
    """Sec. 3.3's second-order accurate interpolation read as trilinear: the sum over
    ALL nodes of product tent weights max(0, 1 - |d|/h) (periodic in x, y)."""
    rng = np.random.default_rng(11)
    nx, ny, nz = 8, 8, 8
    grid = (nx, ny, nz, 1.0, 0.8, 0.7)
    dx, dy, dz = 1.0 / nx, 0.8 / ny, 0.7 / (nz - 1)
    f = rng.standard_normal((nz, ny, nx))
    x, y, z_uv, z_w = inputs.node_coords(grid)

    def tent(d, h, period=None):
        if period is not None:
            d = d - period * np.round(d / period)
        return np.maximum(0.0, 1.0 - np.abs(d) / h)

    for is_w, zlev, top in ((0, z_uv[: nz - 1], nz - 2), (1, z_w, nz - 1)):
        for _ in range(60):
            px = rng.uniform(-1.0, 2.0)
            py = rng.uniform(-1.0, 2.0)
            pz = rng.uniform(zlev[0], zlev[top])
            wx = tent(px - x, dx, 1.0)
            wy = tent(py - y, dy, 0.8)
            wz = tent(pz - zlev, dz)
            brute = np.einsum("k,j,i,kji->", wz, wy, wx, f[: top + 1])
            assert oracle_mod.interp(grid, f, is_w, px, py, pz) == pytest.approx(brute, rel=1e-12, abs=1e-12)
        # clamping: below the lowest and above the highest physical level
        px, py = 0.33, 0.41
        assert oracle_mod.interp(grid, f, is_w, px, py, zlev[0] - 0.3) == pytest.approx(
            oracle_mod.interp(grid, f, is_w, px, py, zlev[0]), rel=1e-14)
        assert oracle_mod.interp(grid, f, is_w, px, py, zlev[top] + 0.5) == pytest.approx(
            oracle_mod.interp(grid, f, is_w, px, py, zlev[top]), rel=1e-14)
        # at a node the interpolant is the node value
        assert oracle_mod.interp(grid, f, is_w, x[3], y[5], zlev[2]) == pytest.approx(f[2, 5, 3], rel=1e-13)


# --------------------------------------------------------------------------- #
# T5: velocity along n gives no stress; tau is homogeneous of degree 2
# --------------------------------------------------------------------------- #
def test_normal_velocity_and_homogeneity(oracle_mod):
    """Sec. 3.3: U_r = u - (u.n)n, so u parallel to n has U_r = 0 and tau = 0;
    tau_w ~ U_r^2 (Eq. 28) with the direction t = U_r/|U_r| makes
    tau(alpha u) = alpha |alpha| tau(u): the stress always opposes the flow."""
    case = inputs.make("ridge", shape=(32, 16, 24), seed=7)
    cu, cw = oracle_mod.classify(case.grid, case.phi_uv, case.phi_w, case.phi_b)
    nw = oracle_mod.normals(case.grid, case.phi_w)
    kk, jj, ii = np.nonzero(cw == 1)
    sel = list(range(0, len(kk), max(1, len(kk) // 12)))
    for s in sel:
        k, j, i = int(kk[s]), int(jj[s]), int(ii[s])
        n = nw[:, k, j, i]
        # uniform velocity along this node's normal
        u = np.full(case.shape, 2.5 * n[0])
        v = np.full(case.shape, 2.5 * n[1])
        w = np.full(case.shape, 2.5 * n[2])
        t, tw, ur = oracle_mod.wall_model_node(case.grid, case.phi_w, 1, i, j, k, u, v, w, 1e-4, case.phi_c)
        assert np.max(np.abs(t)) < 1e-13 and abs(ur) < 1e-13
        # homogeneity on the noisy field
        t1, tw1, _ = oracle_mod.wall_model_node(case.grid, case.phi_w, 1, i, j, k, case.u, case.v, case.w,
                                                1e-4, case.phi_c)
        for a in (-1.7, 0.6):
            t2, tw2, _ = oracle_mod.wall_model_node(case.grid, case.phi_w, 1, i, j, k, a * case.u, a * case.v,
                                                    a * case.w, 1e-4, case.phi_c)
            np.testing.assert_allclose(t2, a * abs(a) * t1, rtol=1e-12, atol=1e-14)
            assert tw2 == pytest.approx(a * a * tw1, rel=1e-12)
        assert np.trace(t1) == pytest.approx(0.0, abs=1e-12)   # t.n = 0 makes tau traceless


def test_z0_outside_range_rejected(oracle_mod):
    case = inputs.flat((8, 8, 9))
    tau = _fresh_tau(case.shape, 0.0)
    with pytest.raises(ValueError):
        oracle_mod.wall_stress(case.grid, case.phi_uv, case.phi_w, 2 * case.phi_c, case.phi_c, case.phi_b,
                               case.u, case.v, case.w, tau)


# --------------------------------------------------------------------------- #
# normals: exact for planes, second order for curved terrain (Sec. 3.1)
# --------------------------------------------------------------------------- #
def test_normals_second_order(oracle_mod):
    """n = grad(phi)/|grad(phi)| for phi = z - h(x) of the Eq. 31 ridge is
    (-h', 0, 1)/sqrt(1 + h'^2); central differences converge at second order."""
    errs = []
    for nx in (64, 128, 256):
        grid = (nx, 4, 9, 2 * math.pi, 1.0, 1.0)
        h = inputs.ridge_height(grid, height=0.1, half_width=0.6)
        phi_uv, _ = inputs.heightfield_phi(grid, h)
        nrm = oracle_mod.normals(grid, phi_uv)
        x = np.arange(nx) * (2 * math.pi / nx)
        xr = x - 0.25 * 2 * math.pi
        b = 0.6
        hp = np.where(np.abs(xr) < b, -0.1 * (math.pi / (2 * b)) * np.sin(math.pi * xr / b), 0.0)
        mag = np.sqrt(1 + hp ** 2)
        k = 4
        # h'' jumps at the ridge foot |x| = b: measure the smooth part only
        smooth = np.abs(np.abs(xr) - b) > 0.1
        errs.append(max(np.max(np.abs(nrm[0, k, 0] + hp / mag)[smooth]),
                        np.max(np.abs(nrm[2, k, 0] - 1 / mag)[smooth])))
        assert np.max(np.abs(nrm[1, k])) == 0.0
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0


# --------------------------------------------------------------------------- #
# T6: the divergence on the staggered grid
# --------------------------------------------------------------------------- #
def _zeros_tau(shape):
    return {k: np.zeros(shape) for k in inputs.TAU_NAMES}


def test_force_constant_and_linear(oracle_mod):
    """Eq. 2: f = -div(tau).  A constant stress has no divergence; tau_xz = a z and
    tau_zz = b z give f_x = -a (Eq. 16 on uv-nodes) and f_z = -b (Eq. 15 on
    interior w-nodes) exactly; boundary rows follow reading R6."""
    nx, ny, nz = 12, 10, 17
    grid = (nx, ny, nz, 1.5, 1.0, 1.0)
    rng = np.random.default_rng(3)
    shape = (nz, ny, nx)
    tau = {k: np.full(shape, rng.uniform(-1, 1)) for k in inputs.TAU_NAMES}
    fx, fy, fz = oracle_mod.force(grid, tau)
    assert np.max(np.abs(fx)) == 0 and np.max(np.abs(fy)) == 0 and np.max(np.abs(fz)) == 0

    _, _, z_uv, z_w = inputs.node_coords(grid)
    a, b, c = 0.75, -1.25, 2.0
    tau = _zeros_tau(shape)
    tau["txz"] = np.ascontiguousarray(np.broadcast_to(a * z_w[:, None, None], shape))
    tau["tyz"] = np.ascontiguousarray(np.broadcast_to(c * z_w[:, None, None], shape))
    tau["tzz"] = np.ascontiguousarray(np.broadcast_to(b * z_uv[:, None, None], shape))
    fx, fy, fz = oracle_mod.force(grid, tau)
    np.testing.assert_allclose(fx[: nz - 1], -a, rtol=1e-12)
    np.testing.assert_allclose(fy[: nz - 1], -c, rtol=1e-12)
    assert np.all(fx[nz - 1] == 0) and np.all(fy[nz - 1] == 0)
    np.testing.assert_allclose(fz[1: nz - 1], -b, rtol=1e-12)
    assert np.all(fz[0] == 0) and np.all(fz[nz - 1] == 0)


@pytest.mark.parametrize("comp,axis", [("txx", "x"), ("txy", "y"), ("txy", "x"), ("tyy", "y"),
                                       ("txz", "x"), ("tyz", "y")])
def test_force_sinusoid(oracle_mod, comp, axis):
    """Central differences of sin(k x) give cos(k x) sin(k h)/h exactly (periodic)."""
    nx, ny, nz = 32, 24, 6
    lx, ly = 2.0, 3.0
    grid = (nx, ny, nz, lx, ly, 1.0)
    shape = (nz, ny, nx)
    x, y, _, _ = inputs.node_coords(grid)
    m = 3
    if axis == "x":
        kw, h, coord = 2 * math.pi * m / lx, lx / nx, x[None, None, :]
    else:
        kw, h, coord = 2 * math.pi * m / ly, ly / ny, y[None, :, None]
    tau = _zeros_tau(shape)
    tau[comp] = np.ascontiguousarray(np.broadcast_to(np.sin(kw * coord), shape))
    fx, fy, fz = oracle_mod.force(grid, tau)
    d = np.broadcast_to(np.cos(kw * coord) * math.sin(kw * h) / h, shape)
    target = {("txx", "x"): ("fx", 0), ("txy", "y"): ("fx", 0), ("txy", "x"): ("fy", 0),
              ("tyy", "y"): ("fy", 0), ("txz", "x"): ("fz", 1), ("tyz", "y"): ("fz", 1)}[(comp, axis)]
    fout = {"fx": fx, "fy": fy, "fz": fz}[target[0]]
    if target[0] == "fz":
        np.testing.assert_allclose(fout[1: nz - 1], -d[1: nz - 1], atol=1e-12)
    else:
        np.testing.assert_allclose(fout[: nz - 1], -d[: nz - 1], atol=1e-12)


def test_force_plane_sums_telescope(oracle_mod):
    """Periodic horizontal differences sum to zero over a plane, so the plane sum of
    f_x is -sum (txz[k+1] - txz[k]) / dz and of f_z is -sum (tzz[k] - tzz[k-1]) / dz."""
    nx, ny, nz = 16, 12, 10
    grid = (nx, ny, nz, 1.0, 1.0, 1.0)
    dz = 1.0 / (nz - 1)
    rng = np.random.default_rng(5)
    tau = {k: rng.standard_normal((nz, ny, nx)) for k in inputs.TAU_NAMES}
    fx, fy, fz = oracle_mod.force(grid, tau)
    for k in range(nz - 1):
        assert fx[k].sum() == pytest.approx(-(tau["txz"][k + 1] - tau["txz"][k]).sum() / dz, rel=1e-10, abs=1e-8)
        assert fy[k].sum() == pytest.approx(-(tau["tyz"][k + 1] - tau["tyz"][k]).sum() / dz, rel=1e-10, abs=1e-8)
    for k in range(1, nz - 1):
        assert fz[k].sum() == pytest.approx(-(tau["tzz"][k] - tau["tzz"][k - 1]).sum() / dz, rel=1e-10, abs=1e-8)


# --------------------------------------------------------------------------- #
# T7: body mask (Sec. 3.2, Eq. 27)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("with_gradp", [False, True])
def test_mask_sets(oracle_mod, with_gradp):
    """Eq. 27: entries with phi <= 0 (on each component's own grid) become
    3 dt/2 grad p (or 0 without a pressure gradient: Sec. 3.2 keeps the body at rest);
    all others are untouched."""
    case = inputs.make("ridge", shape=(32, 8, 16), seed=9)
    rng = np.random.default_rng(1)
    gp = tuple(rng.standard_normal(case.shape) for _ in range(3)) if with_gradp else None
    dt = 0.013
    u, v, w = case.u.copy(), case.v.copy(), case.w.copy()
    oracle_mod.mask(case.grid, case.phi_uv, case.phi_w, u, v, w, gp, dt)
    for new, old, phi, comp in ((u, case.u, case.phi_uv, 0), (v, case.v, case.phi_uv, 1), (w, case.w, case.phi_w, 2)):
        body = phi <= 0
        assert body.any() and (~body).any()
        assert np.array_equal(new[~body], old[~body])
        exp = 1.5 * dt * gp[comp][body] if with_gradp else 0.0
        assert np.array_equal(new[body], np.broadcast_to(exp, new[body].shape))


# --------------------------------------------------------------------------- #
# classes follow the paper's inequalities on a generic terrain
# --------------------------------------------------------------------------- #
def test_classes_partition(oracle_mod):
    """Sec. 3.3: fluid, band and solid partition each grid, and the band is exactly
    the closed interval of the inequalities (checked on the cube array)."""
    case = inputs.make("cubes", shape=(64, 32, 32))
    cu, cw = oracle_mod.classify(case.grid, case.phi_uv, case.phi_w, case.phi_b)
    pb = case.phi_b
    assert np.array_equal(cw == 1, (case.phi_w >= -pb) & (case.phi_w <= pb))
    assert np.array_equal(cw == 2, case.phi_w < -pb)
    assert np.array_equal(cu == 1, (case.phi_uv >= 0) & (case.phi_uv <= 2 * pb))
    assert np.array_equal(cu == 2, case.phi_uv < 0)
    assert (cw == 1).sum() > 0 and (cu == 1).sum() > 0


def test_wall_stress_component_assignment(oracle_mod):
    """Sec. 3.3: tau_xz, tau_yz are modeled at w-band nodes and tau_xx, tau_xy,
    tau_yy, tau_zz at uv-band nodes; checked entry by entry against the hand
    closed form on a tilted plane (interior columns, off the periodic seam)."""
    z0, phi_c = 1e-3, 0.06
    normal, uvec = (0.25, -0.3, 1.0), (1.1, 0.6, -0.2)
    grid, phi_uv, phi_w, u, v, w, nrm = _plane_case(normal, 0.3, uvec)
    nx, ny, nz = grid[:3]
    C = (KAPPA / math.log(phi_c / z0)) ** 2
    tref, twref, _ = _closed_form(nrm, uvec, C)
    tau = _fresh_tau((nz, ny, nx), 5.0)
    pb = 0.5 / (nz - 1)
    stats = oracle_mod.wall_stress(grid, phi_uv, phi_w, z0, phi_c, pb, u, v, w, tau)
    cu, cw = oracle_mod.classify(grid, phi_uv, phi_w, pb)
    inner = np.zeros((nz, ny, nx), bool)
    inner[1:nz - 1, 1:ny - 1, 1:nx - 1] = True
    for name, (a, b) in (("txz", (0, 2)), ("tyz", (1, 2))):
        sel = (cw == 1) & inner
        assert sel.sum() > 10
        np.testing.assert_allclose(tau[name][sel], tref[a, b], rtol=1e-12, atol=1e-13)
        assert np.all(tau[name][cw == 2] == 0.0) and np.all(tau[name][cw == 0] == 5.0)
    for name, (a, b) in (("txx", (0, 0)), ("txy", (0, 1)), ("tyy", (1, 1)), ("tzz", (2, 2))):
        sel = (cu == 1) & inner
        assert sel.sum() > 10
        np.testing.assert_allclose(tau[name][sel], tref[a, b], rtol=1e-12, atol=1e-13)
        assert np.all(tau[name][cu == 2] == 0.0) and np.all(tau[name][cu == 0] == 5.0)
    assert stats[0, 0] == (cw == 1).sum() and stats[1, 0] == (cu == 1).sum()
