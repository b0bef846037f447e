"""GPU signed distance to a height field (wmibm_heightfield_sdf, Sec. 3.1) against
the oracle's brute force over every triangle: whole arrays on small, ragged and
anisotropic grids with narrow and wide reaches, sampled nodes of the full
512 x 256 x 256 hill, the distance properties at full size, degenerate grids
(one column row, reach below a cell), the chain into wmibm_init (node classes
equal to the oracle's on the oracle's distance), and argument checks."""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-12        # FP64 distances of O(0.1): a few hundred ulps of room for the different operation order
EDGE = 1e-9        # nodes this close to the reach may fall on either side of it


@pytest.fixture(scope="module")
def wm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03343_gb300 import build, wmibm
    build.build()
    wmibm.load()
    return wmibm


def _gpu(wm, grid, h, reach):
    ht = torch.from_numpy(np.ascontiguousarray(h, dtype=np.float64)).cuda()
    pu, pw = wm.heightfield_sdf(grid, ht, reach)
    torch.cuda.synchronize()
    return pu.cpu().numpy(), pw.cpu().numpy()


def _vertical(grid, h, is_w):
    _, _, zu, zw = inputs.node_coords(grid)
    z = zw if is_w else zu
    return z[:, None, None] - h[None, :, :]


def _compare(oracle_mod, grid, h, reach, got, nodes=None):
    """Element by element against the oracle, except within EDGE of the reach,
    where the GPU value must be one of the two valid answers."""
    for is_w, g in zip((False, True), got):
        d = oracle_mod.heightfield_distance(grid, h, is_w, nodes)
        vert = _vertical(grid, h, is_w)
        if nodes is not None:
            vert = vert.reshape(-1)[nodes]
            g = g.reshape(-1)[nodes]
        ref = np.where(d <= reach, np.sign(vert) * d, vert)
        edge = np.abs(d - reach) <= EDGE
        assert np.all(np.abs(g[~edge] - ref[~edge]) <= TOL), (is_w, float(np.max(np.abs(g[~edge] - ref[~edge]))))
        if edge.any():
            ok = (np.abs(g[edge] - vert[edge]) <= TOL) | (np.abs(g[edge] - np.sign(vert[edge]) * d[edge]) <= TOL)
            assert ok.all()


def _hills(grid, seed, lift=0.05):
    return inputs.gaussian_hills_height(grid, np.random.default_rng(seed), nhills=4) + lift


CASES = [
    ((24, 20, 16, 1.2, 1.0, 1.0), 0.08),           # isotropic, reach of ~2 cells
    ((13, 7, 9, 1.3, 0.7, 0.5), 0.12),             # ragged column count (one partial block), reach > a cell
    ((40, 12, 20, 2.0, 1.2, 1.0), 0.02),           # dy = 2 dx, reach below one cell
    ((16, 16, 33, 1.0, 1.0, 1.0), 0.2),            # wide window: 8 x 8 cells
]


@pytest.mark.parametrize("grid,reach", CASES)
def test_sdf_matches_oracle(wm, oracle_mod, grid, reach):
    nx, ny = grid[0], grid[1]
    h = _hills(grid, seed=nx * 31 + ny)
    _compare(oracle_mod, grid, h, reach, _gpu(wm, grid, h, reach))


def test_sdf_wide_window_and_tall_grid(wm, oracle_mod):
    """A reach of 15 cells (the heights no longer fit the block's shared tiles, so
    they come from global memory) and 1300 levels (the z table no longer fits)."""
    grid = (64, 40, 14, 1.0, 0.625, 1.0)
    h = _hills(grid, seed=21)
    _compare(oracle_mod, grid, h, 15.0 / 64, _gpu(wm, grid, h, 15.0 / 64))
    grid = (8, 6, 1300, 1.0, 0.75, 1.0)
    h = _hills(grid, seed=22)
    _compare(oracle_mod, grid, h, 0.1, _gpu(wm, grid, h, 0.1))


def test_sdf_tents_and_spike(wm, oracle_mod):
    """Surfaces with creases on grid lines (the diagonal tent follows the split
    diagonal) and a single-vertex spike, whose nearest points are edges and vertices."""
    n, L = 24, 1.5
    grid = (n, n, 20, L, L, 1.0)
    x = np.arange(n) * (L / n)
    u = x[None, :] - x[:, None]
    um = u - L * np.round(u / L)
    _compare(oracle_mod, grid, np.maximum(0.0, 0.125 - 0.5 * np.abs(um)), 0.15,
             _gpu(wm, grid, np.maximum(0.0, 0.125 - 0.5 * np.abs(um)), 0.15))
    grid = (20, 20, 16, 2.0, 2.0, 1.0)
    spike = np.zeros((20, 20))
    spike[12, 8] = 0.3
    _compare(oracle_mod, grid, spike, 0.45, _gpu(wm, grid, spike, 0.45))


def test_sdf_full_size_hill(wm, oracle_mod):
    """The 512 x 256 x 256 hill (Eq. 32) at reach 4 dz: every node near the surface
    that the oracle can afford (sampled), and the properties of a distance everywhere."""
    grid = (512, 256, 256, 2 * np.pi, np.pi, 1.0)
    h = inputs.hill_height(grid)
    dz = 1.0 / 255
    reach = 4 * dz
    got = _gpu(wm, grid, h, reach)
    rng = np.random.default_rng(9)
    near = np.flatnonzero(np.abs(_vertical(grid, h, True)).reshape(-1) <= 6 * dz)
    _compare(oracle_mod, grid, h, reach, got, np.sort(rng.choice(near, size=400, replace=False)))
    for is_w, g in zip((False, True), got):
        vert = _vertical(grid, h, is_w)
        assert np.all(np.sign(g) == np.sign(vert))
        assert np.all(np.abs(g) <= np.abs(vert) + TOL)
        far = np.abs(g) > reach
        assert np.array_equal(g[far], vert[far])
        # 1-Lipschitz between vertical neighbours where both are exact
        both = (np.abs(g[1:]) <= reach) & (np.abs(g[:-1]) <= reach)
        assert np.all(np.abs(np.diff(g, axis=0))[both] <= dz + TOL)
        shorter = np.abs(g) < np.abs(vert) - 1e-6
        assert shorter.any()                                       # the slopes do shorten the distance


def test_sdf_single_row_equals_constant_in_y(wm):
    """ny = 1: the window wraps onto the one row many times over; a ridge constant
    in y must give the same distance as on a 4-row grid."""
    g4 = (32, 4, 12, 1.0, 0.4, 0.5)
    g1 = (32, 1, 12, 1.0, 0.1, 0.5)
    h1 = inputs.ridge_height(g4, height=0.1, half_width=0.3)[0]
    a = _gpu(wm, g4, np.tile(h1, (4, 1)), 0.06)
    b = _gpu(wm, g1, h1[None, :], 0.06)
    for x, y in zip(a, b):
        for j in range(4):
            assert np.allclose(x[:, j, :], y[:, 0, :], atol=TOL, rtol=0)


def test_sdf_flat_is_vertical(wm):
    grid = (33, 17, 10, 1.0, 0.5, 1.0)
    h = np.full((17, 33), 0.31)
    for g, is_w in zip(_gpu(wm, grid, h, 0.1), (False, True)):
        assert np.allclose(g, _vertical(grid, h, is_w), atol=1e-15, rtol=0)


def test_sdf_then_init_classes_match_oracle(wm, oracle_mod):
    """The GPU distance fed to wmibm_init gives the node classes the oracle gives on
    its own distance (no node sits within 1e-9 of a class threshold here)."""
    grid = (64, 32, 24, 2.0, 1.0, 1.0)
    h = _hills(grid, seed=5, lift=0.08)
    dz = 1.0 / 23
    phi_b = 0.5 * dz
    pu, pw = _gpu(wm, grid, h, 3 * dz)
    ou, ow = oracle_mod.heightfield_sdf(grid, h, 3 * dz)
    for a in (ou, ow):
        for t in (0.0, phi_b, 2 * phi_b, -phi_b):
            assert np.min(np.abs(a - t)) > 1e-9
    h_ = wm.Handle(grid, pu, pw, 1e-4, 1.5 * dz, phi_b=phi_b, dtype="f64")
    cu, cw = oracle_mod.classify(grid, ou, ow, phi_b)
    expect = {wm.LIST_BAND_W: np.flatnonzero(cw.reshape(-1) == 1), wm.LIST_BAND_UV: np.flatnonzero(cu.reshape(-1) == 1),
              wm.LIST_SOLID_W: np.flatnonzero(cw.reshape(-1) == 2),
              wm.LIST_SOLID_UV: np.flatnonzero(cu.reshape(-1) == 2)}
    for which, idx in expect.items():
        assert np.array_equal(h_.export_list(which), idx), which


def test_sdf_rejects_bad_arguments(wm):
    grid = (8, 8, 6, 1.0, 1.0, 1.0)
    h = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    for reach, msg in ((0.0, "reach"), (float("nan"), "reach"), (float("inf"), "reach"), (20.0, "window")):
        with pytest.raises(wm.WmibmError, match=msg):
            wm.heightfield_sdf(grid, h, reach)
    with pytest.raises(wm.WmibmError, match="sizes"):
        wm.heightfield_sdf((8, 8, 2, 1.0, 1.0, 1.0), h, 0.1)
    same = torch.empty((6, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(wm.WmibmError, match="distinct"):
        wm.heightfield_sdf(grid, h, 0.1, phi_uv=same, phi_w=same)
    with pytest.raises(ValueError):
        wm.heightfield_sdf(grid, h.float(), 0.1)
