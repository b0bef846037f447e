"""GPU pseudo-spectral forcing (wmibm_force_spectral: x and y derivatives by
Eqs. 13-14, vertical differences by Eqs. 15-16) against the FP64 oracle's
force_spectral on the same seeded stresses: small grids that span several row
and column units, several level chunks and the edge sizes (2-point lines, the
longest lines (2048 points FP32, 1024 FP64), every radix sequence of the FP32
passes (16, 16 x 8, 16 x 16, 16 x 8 x 8, 16 x 16 x 8), nx < ny and nx > ny); the
full 512 x 256 x 256 hill grid on
sampled levels; graph replay; determinism; and the stage a1 + spectral a2
against the oracle's wall stress followed by its spectral divergence."""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import TOL, normwise, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03343_gb300 import build, wmibm
    build.build()
    wmibm.load()
    return wmibm


def _random_tau(shape, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    return {k: scale * rng.standard_normal(shape) for k in inputs.TAU_NAMES}


def _handle(wm, shape, dtype, lengths=(2 * np.pi, np.pi, 1.0)):
    case = inputs.flat(shape, wall_height=0.3 * lengths[2] / (shape[2] - 1) + 0.0, lengths=lengths)
    return wm.Handle.from_case(case, dtype=dtype), case.grid


def _gpu_spectral(h, tau, dtype):
    shp = h.shape
    t = [to_dev(tau[k], dtype) for k in inputs.TAU_NAMES]
    f = [torch.full(shp, float("nan"), dtype=h.torch_dtype, device="cuda") for _ in range(3)]
    h.force_spectral(t, f)
    torch.cuda.synchronize()
    return [to_host(x) for x in f], t


def _rounded(tau, dtype):
    return {k: to_host(to_dev(v, dtype)) for k, v in tau.items()}


SMALL = [((64, 32, 12), "f32"), ((64, 32, 12), "f64"), ((32, 16, 9), "f32"), ((16, 64, 5), "f64"),
         ((128, 8, 6), "f32"), ((2, 2, 3), "f32"), ((2, 2, 3), "f64"), ((4, 128, 4), "f32"),
         ((256, 2, 3), "f64")]


@pytest.mark.parametrize("shape,dtype", SMALL)
def test_spectral_force_matches_oracle(wm, oracle_mod, shape, dtype):
    h, grid = _handle(wm, shape, dtype)
    nx, ny, nz = shape
    tau = _random_tau((nz, ny, nx), seed=nx * 7 + ny + nz)
    got, _ = _gpu_spectral(h, tau, dtype)
    ref = oracle_mod.force_spectral(grid, _rounded(tau, dtype))
    for c in range(3):
        assert np.all(np.isfinite(got[c]))
        err = normwise(got[c], ref[c])[0]
        assert err <= TOL[dtype], (c, err)
    assert np.all(got[0][-1] == 0) and np.all(got[1][-1] == 0)
    assert np.all(got[2][0] == 0) and np.all(got[2][-1] == 0)
    assert h.device_status() == wm.OK


@pytest.mark.parametrize("shape,dtype", [((512, 256, 12), "f32"), ((512, 256, 8), "f64"), ((2048, 4, 3), "f32"),
                                         ((8, 2048, 3), "f32"), ((1024, 8, 3), "f64"), ((4, 1024, 3), "f64"),
                                         ((1024, 16, 3), "f32"), ((16, 1024, 3), "f32")])
def test_spectral_force_several_chunks_and_longest_lines(wm, oracle_mod, shape, dtype):
    """Grids whose level chunks are fewer than the levels (the column units wait on
    row units of earlier chunks) and the longest lines in either direction (2048
    points in FP32, 1024 in FP64)."""
    h, grid = _handle(wm, shape, dtype)
    rx, wy, kc, smem = h.spectral_shape()
    nx, ny, nz = shape
    assert ny % rx == 0 and nx % wy == 0 and 1 <= kc <= nz and smem <= 227 * 1024
    tau = _random_tau((nz, ny, nx), seed=17)
    got, _ = _gpu_spectral(h, tau, dtype)
    ref = oracle_mod.force_spectral(grid, _rounded(tau, dtype))
    for c in range(3):
        assert normwise(got[c], ref[c])[0] <= TOL[dtype], c
    assert h.device_status() == wm.OK


def test_spectral_force_single_modes_exact(wm):
    """A stress made of single Fourier modes below Nyquist: the FP64 GPU forcing
    equals the analytic -div tau (closed form, no oracle) to rounding."""
    nx, ny, nz = 64, 32, 6
    lx, ly, lz = 2 * np.pi, np.pi, 1.0
    h, grid = _handle(wm, (nx, ny, nz), "f64", (lx, ly, lz))
    x, y, z_uv, z_w = inputs.node_coords(grid)
    X, Y = x[None, None, :], y[None, :, None]
    Zw = z_w[:, None, None]
    kx, ky = 2 * np.pi * 5 / lx, 2 * np.pi * 3 / ly
    shp = (nz, ny, nx)
    b = lambda a: np.ascontiguousarray(np.broadcast_to(a, shp))
    tau = dict(txx=b(np.sin(kx * X + ky * Y)), txy=b(np.cos(kx * X - ky * Y)), tyy=b(np.sin(ky * Y)),
               tzz=b(0 * X), txz=b(2.0 * Zw + 0 * X + np.cos(kx * X)), tyz=b(0 * Zw + np.sin(2 * ky * Y)))
    got, _ = _gpu_spectral(h, tau, "f64")
    fx = -(kx * np.cos(kx * X + ky * Y) + ky * np.sin(kx * X - ky * Y) + 2.0)
    fy = -(-kx * np.sin(kx * X - ky * Y) + ky * np.cos(ky * Y))
    fz = -(-kx * np.sin(kx * X) + 2 * ky * np.cos(2 * ky * Y))
    for g, r in ((got[0][:-1], b(fx)[:-1]), (got[1][:-1], b(fy)[:-1]), (got[2][1:-1], b(fz)[1:-1])):
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()


def test_full_size_hill_sampled_levels(wm, oracle_mod):
    """The 512 x 256 x 256 hill grid in FP32 (the spectral bench workload) with its
    seeded fluid stresses: levels 0, 1, 100, 254 and 255 against the oracle.  A
    level needs only its own plane and the planes next to it, so the oracle runs
    on the three-level slab k-1..k+1 (a grid of lz = 2 dz)."""
    case = inputs.hill(dtype="f32")
    h = wm.Handle.from_case(case, dtype="f32")
    got, _ = _gpu_spectral(h, case.tau, "f32")
    nx, ny, nz, lx, ly, lz = case.grid
    dz = lz / (nz - 1)
    rt = _rounded(case.tau, "f32")
    for k in (1, 100, 254):
        slab = {n: np.ascontiguousarray(v[k - 1:k + 2]) for n, v in rt.items()}
        ref = oracle_mod.force_spectral((nx, ny, 3, lx, ly, 2 * dz), slab)
        for c in range(3):
            assert normwise(got[c][k], ref[c][1])[0] <= TOL["f32"], (k, c)
    # floor: f_x, f_y of level 0 from the slab 0..2 (level 0 is interior for them); f_z = 0 there
    slab = {n: np.ascontiguousarray(v[0:3]) for n, v in rt.items()}
    ref = oracle_mod.force_spectral((nx, ny, 3, lx, ly, 2 * dz), slab)
    for c in range(2):
        assert normwise(got[c][0], ref[c][0])[0] <= TOL["f32"], c
    assert np.all(got[2][0] == 0)
    assert np.all(got[0][-1] == 0) and np.all(got[1][-1] == 0) and np.all(got[2][-1] == 0)
    assert h.device_status() == wm.OK


def test_spectral_graph_replay_and_determinism(wm):
    """Captured once and replayed: every replay gives the eager result bit for bit
    (the launch re-arms its counters), and two eager calls agree bit for bit."""
    shape = (256, 128, 24)
    h, grid = _handle(wm, shape, "f32")
    tau = _random_tau((24, 128, 256), seed=4)
    a, t = _gpu_spectral(h, tau, "f32")
    b, _ = _gpu_spectral(h, tau, "f32")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    f = [torch.zeros(h.shape, dtype=torch.float32, device="cuda") for _ in range(3)]
    h.force_spectral(t, f)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h.force_spectral(t, f)
    for _ in range(5):
        for x in f:
            x.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for x, y in zip(f, a):
            assert np.array_equal(to_host(x), y)
    for x, name in zip(t, inputs.TAU_NAMES):                 # the stresses are read only
        assert np.array_equal(to_host(x), to_host(to_dev(tau[name], "f32")))
    assert h.device_status() == wm.OK


def test_unsupported_grid_is_rejected(wm):
    """nx or ny not a power of two, or FP64 lines longer than 1024 points: EINVAL
    with a message, nothing launched."""
    h, grid = _handle(wm, (48, 32, 5), "f32")
    assert h.spectral_shape() is None
    tau = [torch.zeros(h.shape, dtype=torch.float32, device="cuda") for _ in range(6)]
    f = [torch.zeros(h.shape, dtype=torch.float32, device="cuda") for _ in range(3)]
    with pytest.raises(wm.WmibmError, match="power"):
        h.force_spectral(tau, f)
    h64, _ = _handle(wm, (2048, 4, 3), "f64")              # FP64 lines stop at 1024 points
    assert h64.spectral_shape() is None
    tau = [torch.zeros(h64.shape, dtype=torch.float64, device="cuda") for _ in range(6)]
    f = [torch.zeros(h64.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(wm.WmibmError, match="power"):
        h64.force_spectral(tau, f)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_wall_stress_then_spectral_force_matches_oracle(wm, oracle_mod, dtype):
    """The stage with the paper's horizontal scheme: GPU wall stress (a1) then the
    spectral divergence (a2) on the ridge terrain, against the oracle's wall stress
    followed by its spectral divergence on the same rounded inputs."""
    case = inputs.ridge(shape=(64, 32, 32), dtype=dtype)
    h = wm.Handle.from_case(case, dtype=dtype)
    u, v, w = (to_dev(x, dtype) for x in (case.u, case.v, case.w))
    tau = [to_dev(case.tau[k], dtype) for k in inputs.TAU_NAMES]
    f = [torch.zeros(h.shape, dtype=h.torch_dtype, device="cuda") for _ in range(3)]
    h.wall_stress(u, v, w, tau)
    h.force_spectral(tau, f)
    torch.cuda.synchronize()
    rd = lambda a: to_host(to_dev(a, dtype))
    tau_o = {k: rd(case.tau[k]) for k in inputs.TAU_NAMES}
    oracle_mod.wall_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b,
                           rd(case.u), rd(case.v), rd(case.w), tau_o)
    f_o = oracle_mod.force_spectral(case.grid, tau_o)
    for k, t in zip(inputs.TAU_NAMES, tau):
        assert normwise(to_host(t), tau_o[k])[0] <= TOL[dtype], k
    for c in range(3):
        assert normwise(to_host(f[c]), f_o[c])[0] <= TOL[dtype], c
    assert h.device_status() == wm.OK
