"""The paper's flat-terrain cases (Sec. 4.1) from the committed fixture
tests/golden/flat_terrain_sec4_1.txt: on both printed grids, the oracle's node
classes are the hand-derived levels, and with the log law of Eq. 29 (u* = 1,
the printed z0) every w-band node carries tau_xz = <tau_w> = -1 and every
uv-band node zero stress, as the paper's set-up prescribes."""
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    params, grids, cases = {}, [], []
    with open(os.path.join(HERE, "golden", "flat_terrain_sec4_1.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "grid":
                grids.append(tuple(int(v) for v in vals))
            elif key == "case":
                sets = [set() if v == "-" else {int(x) for x in v.split(",")} for v in vals[1:5]]
                cases.append((float(vals[0]), *sets, float(vals[5])))
            else:
                params[key] = float(vals[0])
    return params, grids, cases


PARAMS, GRIDS, CASES = _load()


def _fields(grid_shape, c, phi_c_cells):
    nx, ny, nz = grid_shape
    lx, ly, lz = PARAMS["lx"], PARAMS["ly"], PARAMS["lz"]
    dz = lz / (nz - 1)
    zw = c * dz
    z_uv = (np.arange(nz) + 0.5) * dz
    z_w = np.arange(nz) * dz
    shp = (nz, ny, nx)
    phi_uv = np.ascontiguousarray(np.broadcast_to((z_uv - zw)[:, None, None], shp))
    phi_w = np.ascontiguousarray(np.broadcast_to((z_w - zw)[:, None, None], shp))
    z0, kappa, ustar = PARAMS["z0"], PARAMS["kappa"], PARAMS["ustar"]
    prof = np.where(phi_uv > z0, (ustar / kappa) * np.log(np.maximum(phi_uv, z0) / z0), 0.0)
    u = np.ascontiguousarray(prof)
    v = np.zeros(shp)
    w = np.zeros(shp)
    return (nx, ny, nz, lx, ly, lz), phi_uv, phi_w, u, v, w, phi_c_cells * dz, 0.5 * dz


def test_fixture_has_the_printed_cases():
    assert [c[0] for c in CASES] == [1.0, 1.25, 1.5, 1.75]
    assert GRIDS == [(64, 32, 33), (256, 128, 129)]
    assert PARAMS["lx"] / PARAMS["lz"] == 8.0 and PARAMS["ly"] / PARAMS["lz"] == 4.0


@pytest.mark.parametrize("grid_shape", GRIDS)
@pytest.mark.parametrize("case", CASES, ids=[f"zw{c[0]}" for c in CASES])
def test_classes_and_wall_stress_of_the_printed_cases(oracle_mod, grid_shape, case):
    c, w_band, w_solid, uv_band, uv_solid, phi_c_cells = case
    grid, phi_uv, phi_w, u, v, w, phi_c, phi_b = _fields(grid_shape, c, phi_c_cells)
    cu, cw = oracle_mod.classify(grid, phi_uv, phi_w, phi_b)
    for cls, band, solid in ((cw, w_band, w_solid), (cu, uv_band, uv_solid)):
        assert {int(k) for k in np.unique(np.nonzero(cls == 1)[0])} == band
        assert {int(k) for k in np.unique(np.nonzero(cls == 2)[0])} == solid
    tau = {k: np.full(u.shape, 0.25) for k in ("txx", "txy", "tyy", "tzz", "txz", "tyz")}
    stats = oracle_mod.wall_stress(grid, phi_uv, phi_w, PARAMS["z0"], phi_c, phi_b, u, v, w, tau,
                                   kappa=PARAMS["kappa"])
    for k in sorted(w_band):
        np.testing.assert_allclose(tau["txz"][k], PARAMS["tau_w"], rtol=1e-12)
        np.testing.assert_allclose(tau["tyz"][k], 0.0, atol=1e-12)
    for k in sorted(uv_band):
        for name in ("txx", "txy", "tyy", "tzz"):
            np.testing.assert_allclose(tau[name][k], 0.0, atol=1e-12)
    nwb = len(w_band) * grid_shape[0] * grid_shape[1]
    assert stats[0, 0] == nwb
    assert math.isclose(stats[0, 1] / nwb, PARAMS["tau_w"], rel_tol=1e-12)     # <tau_w> = -1
