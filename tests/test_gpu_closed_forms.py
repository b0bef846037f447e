"""The GPU stage on inputs whose answer the paper and the mathematics fix, and on
the edges of the interpolation: the flat-wall log law (Sec. 2.3, Eqs. 9-10 and
29), velocity along the normal (Sec. 3.3: U_r = 0 gives no stress), sample
points beyond the top physical level (reading R3: clamped and counted, or
rejected at init), and the entry point without device allocation against the
oracle itself.  Outputs start as NaN where the stage writes them."""
import math

import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import TOL, assert_stats_close, normwise, oracle_step, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KAPPA = 0.4


@pytest.fixture(scope="module")
def wm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03343_gb300 import build, wmibm
    build.build()
    wmibm.load()
    return wmibm


def _flat_case(shape, h, u, v, w, phi_c_cells=1.5, lengths=(1.0, 1.0, 1.0)):
    """Flat terrain at height h with the given velocity fields (phi = z - h)."""
    nx, ny, nz = shape
    dz = lengths[2] / (nz - 1)
    z_uv = (np.arange(nz) + 0.5) * dz
    z_w = np.arange(nz) * dz
    phi_uv = np.ascontiguousarray(np.broadcast_to((z_uv - h)[:, None, None], (nz, ny, nx)))
    phi_w = np.ascontiguousarray(np.broadcast_to((z_w - h)[:, None, None], (nz, ny, nx)))
    tau = {k: np.zeros((nz, ny, nx)) for k in inputs.TAU_NAMES}
    return inputs.Case("flat", (nx, ny, nz) + tuple(lengths), phi_uv, phi_w, 1e-4, phi_c_cells * dz, 0.5 * dz,
                       np.ascontiguousarray(u), np.ascontiguousarray(v), np.ascontiguousarray(w), tau)


def _run(wm, case, dtype, entry="wall_stress_force", zclamp=0):
    h = wm.Handle.from_case(case, dtype=dtype, zclamp=zclamp)
    u, v, w = (to_dev(x, dtype) for x in (case.u, case.v, case.w))
    tau = []
    for k in inputs.TAU_NAMES:
        a = case.tau[k].copy()
        phi = case.phi_w if inputs.TAU_ON_W[k] else case.phi_uv
        a[phi <= (case.phi_b if inputs.TAU_ON_W[k] else 2 * case.phi_b)] = np.nan
        tau.append(to_dev(a, dtype))
    f = [to_dev(np.full(case.shape, np.nan), dtype) for _ in range(3)]
    st = h.new_stats()
    if entry == "wall_stress_force":
        h.wall_stress_force(u, v, w, tau, f, st)
    elif entry == "noalloc":
        h.wall_stress_noalloc(u, v, w, tau, st)
    else:
        h.wall_stress(u, v, w, tau, st)
    torch.cuda.synchronize()
    out = ({k: to_host(t) for k, t in zip(inputs.TAU_NAMES, tau)}, [to_host(t) for t in f], h.parse_stats(st))
    assert h.device_status() == wm.OK
    h.close()
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("theta", [0.0, 0.7])
@pytest.mark.parametrize("entry", ["wall_stress", "wall_stress_force"])
def test_flat_wall_log_law(wm, dtype, theta, entry):
    """Sec. 2.3 Eqs. 9-10 and Eq. 29: u = (u*/kappa) ln(z/z0) along direction theta,
    the sample point on a uv-node (phi_c = 1.5 dz): tau_xz = -u*^2 cos(theta),
    tau_yz = -u*^2 sin(theta) at every w-band node, and no uv-band stress."""
    nx, ny, nz = 16, 8, 33
    dz = 1.0 / 32
    ustar = 1.3
    z_uv = (np.arange(nz) + 0.5) * dz
    prof = (ustar / KAPPA) * np.log(z_uv / 1e-4)
    shape = (nz, ny, nx)
    u = np.broadcast_to((prof * math.cos(theta))[:, None, None], shape)
    v = np.broadcast_to((prof * math.sin(theta))[:, None, None], shape)
    case = _flat_case((nx, ny, nz), 0.0, u, v, np.zeros(shape))
    tau, f, st = _run(wm, case, dtype, entry)
    tol = 1e-12 if dtype == "f64" else 2e-6
    np.testing.assert_allclose(tau["txz"][0], -ustar ** 2 * math.cos(theta), rtol=tol, atol=tol)
    np.testing.assert_allclose(tau["tyz"][0], -ustar ** 2 * math.sin(theta), rtol=tol, atol=tol)
    for name in ("txx", "txy", "tyy", "tzz"):
        np.testing.assert_allclose(tau[name][0], 0.0, atol=tol)
    assert st[0]["count"] == nx * ny and st[1]["count"] == nx * ny
    assert st[0]["n_zclamped"] == 0 and st[1]["n_zclamped"] == 0
    assert st[0]["min_tw"] == pytest.approx(-ustar ** 2, rel=tol)
    if entry == "wall_stress_force":
        # f_x on the first uv-level: -(txz[1] - txz[0]) / dz with txz[1] = 0 (fluid, given as 0)
        np.testing.assert_allclose(f[0][0], -(0.0 + ustar ** 2 * math.cos(theta)) / dz, rtol=tol)
        assert np.all(np.isfinite(f[0])) and np.all(np.isfinite(f[2]))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_velocity_along_the_normal_gives_no_stress(wm, dtype):
    """Sec. 3.3: U_r = u - (u.n)n vanishes for u along n, and so does tau (flat wall,
    n = (0,0,1) exactly: the result is exactly zero in any precision)."""
    nx, ny, nz = 16, 8, 17
    shape = (nz, ny, nx)
    case = _flat_case((nx, ny, nz), 0.21, np.zeros(shape), np.zeros(shape), np.full(shape, 2.5))
    tau, _, st = _run(wm, case, dtype, "wall_stress")
    for name in inputs.TAU_NAMES:
        band = (case.phi_w if inputs.TAU_ON_W[name] else case.phi_uv) <= (
            case.phi_b if inputs.TAU_ON_W[name] else 2 * case.phi_b)
        assert np.all(tau[name][band] == 0.0), name
    for b in range(2):
        assert st[b]["max_ur"] == 0.0 and st[b]["sum_tw"] == 0.0


@pytest.mark.parametrize("above", [False, True])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_sample_points_beyond_the_lid(wm, oracle_mod, dtype, above):
    """Reading R3: a flat wall so high that every band node's sample point h + phi_c
    lies above the top physical uv-level ((nz - 1.5) dz): the level is clamped, the
    result matches the oracle, and every band node is counted in n_zclamped (none
    when the wall sits 0.2 dz lower than that)."""
    nx, ny, nz = 16, 8, 17
    dz = 1.0 / (nz - 1)
    h = (nz - 1.5) * dz - 1.5 * dz + (0.2 if above else -0.2) * dz
    rng = np.random.default_rng(5)
    shape = (nz, ny, nx)
    case = _flat_case((nx, ny, nz), h, rng.standard_normal(shape), rng.standard_normal(shape),
                      rng.standard_normal(shape))
    for k in inputs.TAU_NAMES:
        case.tau[k] = rng.standard_normal(shape)
    tau_g, f_g, st_g = _run(wm, case, dtype)
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    for k in inputs.TAU_NAMES:
        assert normwise(tau_g[k], tau_o[k])[0] <= TOL[dtype], k
    for c in range(3):
        assert normwise(f_g[c], f_o[c])[0] <= TOL[dtype], c
    assert_stats_close(st_g, st_o, dtype)
    for b in range(2):
        assert st_g[b]["n_zclamped"] == (st_g[b]["count"] if above else 0)
    # the same geometry with zclamp = REJECT fails at init exactly when a point is clamped
    if above:
        with pytest.raises(wm.WmibmError) as e:
            wm.Handle.from_case(case, dtype=dtype, zclamp=wm.ZCLAMP_REJECT)
        assert e.value.status == wm.EINVAL
    else:
        wm.Handle.from_case(case, dtype=dtype, zclamp=wm.ZCLAMP_REJECT).close()


@pytest.mark.parametrize("name", ["cubes_small", "hill_ragged", "ridge32"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_entry_against_the_oracle(wm, oracle_mod, name, dtype):
    """wmibm_wall_stress_noalloc (reduction scratch in a static device array) against
    the oracle's wall stress, band and solid entries poisoned with NaN first."""
    case = {"cubes_small": lambda: inputs.cubes(shape=(72, 40, 36)),
            "hill_ragged": lambda: inputs.hill(shape=(98, 50, 40)),
            "ridge32": lambda: inputs.ridge()}[name]()
    tau_g, _, st_g = _run(wm, case, dtype, "noalloc")
    tau_o, _, st_o = oracle_step(oracle_mod, case)
    for k in inputs.TAU_NAMES:
        assert np.all(np.isfinite(tau_g[k])), k
        assert normwise(tau_g[k], tau_o[k])[0] <= TOL[dtype], k
    assert_stats_close(st_g, st_o, dtype)


def test_noalloc_rejects_bands_beyond_its_limit(wm):
    """More than 1,048,576 band nodes: the entry point without allocation returns
    EINVAL before any GPU work (a flat wall at 1.5 dz puts four band nodes in each of
    1024 x 264 columns), while wmibm_wall_stress takes the same band."""
    case = inputs.flat((1024, 264, 8), wall_height=1.5 / 7, lengths=(8.0, 4.0, 1.0), sigma=0.1, seed=4,
                       dtype="f32")
    h = wm.Handle.from_case(case, dtype="f32")
    assert h.list_size(wm.LIST_BAND_W) + h.list_size(wm.LIST_BAND_UV) > 1048576
    u, v, w = (to_dev(x, "f32") for x in (case.u, case.v, case.w))
    tau = [to_dev(case.tau[k], "f32") for k in inputs.TAU_NAMES]
    with pytest.raises(wm.WmibmError) as e:
        h.wall_stress_noalloc(u, v, w, tau)
    assert e.value.status == wm.EINVAL and "1048576" in str(e.value)
    h.wall_stress(u, v, w, tau)
    torch.cuda.synchronize()
    assert h.device_status() == wm.OK
    h.close()
