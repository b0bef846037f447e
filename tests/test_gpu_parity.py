"""GPU parity of the CUDA stress stage against the FP64 oracle, through the C ABI.

Tolerances (normwise, max |gpu - oracle| / max |oracle| per array): 1e-12 for
the FP64 path and 1e-5 for the FP32 path; index lists are compared bit-exactly;
band statistics to 1e-11 (FP64) / 1e-5 (FP32) relative.
"""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import (TOL, assert_stats_close, gpu_step, normwise, oracle_lists, oracle_step, rounded,
                         to_dev, to_host)

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


CASES = {
    "ridge32": lambda: inputs.ridge(),
    "ridge_ragged": lambda: inputs.ridge(shape=(46, 18, 21), seed=21),
    "cubes_small": lambda: inputs.cubes(shape=(72, 40, 36)),
    "hill_ragged": lambda: inputs.hill(shape=(98, 50, 40)),
    "raised_tie": lambda: inputs.flat((64, 32, 33), wall_height=1.5 / 32, lengths=(8.0, 4.0, 1.0), sigma=0.2,
                                      seed=3),
    "ensemble0": lambda: inputs.ensemble_member(0, shape=(64, 64, 64)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_lists_bit_exact(wm, oracle_mod, name):
    """Sec. 3.3 node classes and Eq. 27 body sets: identical ascending lists."""
    case = CASES[name]()
    h = wm.Handle.from_case(case, dtype="f32")
    ref = oracle_lists(oracle_mod, case)
    for which in range(6):
        got = h.export_list(which)
        assert got.dtype == np.int32
        assert np.array_equal(got.astype(np.int64), ref[which]), (name, wm.LIST_NAMES[which])
    h.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_stress_and_force_parity(wm, oracle_mod, name, dtype):
    case = CASES[name]()
    h = wm.Handle.from_case(case, dtype=dtype)
    tau_g, f_g, st_g, _ = gpu_step(h, case, dtype)
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    for k in inputs.TAU_NAMES:
        e, _ = normwise(tau_g[k], tau_o[k])
        assert e <= TOL[dtype], (name, k, e)
    for c in range(3):
        e, _ = normwise(f_g[c], f_o[c])
        assert e <= TOL[dtype], (name, "f" + "xyz"[c], e)
    assert_stats_close(st_g, st_o, dtype)
    h.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_force_alone_same_inputs(wm, oracle_mod, dtype):
    """The divergence kernel on identical (dtype-rounded) stresses: only the
    arithmetic differs, on a ragged grid and on a float4-aligned one."""
    for shape in ((50, 22, 13), (64, 40, 17)):
        case = inputs.hill(shape=shape, seed=31)
        rng = np.random.default_rng(4)
        tau = {k: rounded(rng.standard_normal(case.shape), dtype) for k in inputs.TAU_NAMES}
        h = wm.Handle.from_case(case, dtype=dtype)
        td = [to_dev(tau[k], dtype) for k in inputs.TAU_NAMES]
        f = [to_dev(np.zeros(case.shape), dtype) for _ in range(3)]
        h.force(td, f)
        ref = oracle_mod.force(case.grid, tau)
        for c in range(3):
            e, _ = normwise(to_host(f[c]), ref[c])
            assert e <= (1e-14 if dtype == "f64" else 2e-7), (shape, c, e)
        h.close()


def test_misaligned_buffers_take_scalar_path(wm, oracle_mod):
    case = inputs.cubes(shape=(64, 32, 24))
    h = wm.Handle.from_case(case, dtype="f32")
    tau_g, f_g, st_g, _ = gpu_step(h, case, "f32", offset=1)
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    for c in range(3):
        assert normwise(f_g[c], f_o[c])[0] <= TOL["f32"]
    assert_stats_close(st_g, st_o, "f32")


def test_bf16_velocity_storage(wm, oracle_mod):
    """BF16 velocity storage with FP32 arithmetic: gated against the oracle fed the
    same bf16-rounded velocities; the error against the unrounded velocities is
    only reported."""
    case = inputs.hill(shape=(96, 48, 40))
    h = wm.Handle.from_case(case, dtype="f32", vel_dtype="bf16")
    tau_g, f_g, st_g, _ = gpu_step(h, case, "f32", vel_dtype="bf16")
    ub, vb, wb = (rounded(x, "bf16") for x in (case.u, case.v, case.w))
    tau_o, f_o, st_o = oracle_step(oracle_mod, case, ub, vb, wb)
    for c in range(3):
        assert normwise(f_g[c], f_o[c])[0] <= TOL["f32"]
    for k in inputs.TAU_NAMES:
        assert normwise(tau_g[k], tau_o[k])[0] <= TOL["f32"]
    assert_stats_close(st_g, st_o, "f32")
    tau_x, f_x, _ = oracle_step(oracle_mod, case)
    print("bf16 storage vs unrounded oracle:", [normwise(f_g[c], f_x[c])[0] for c in range(3)])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("with_gradp", [False, True])
def test_mask(wm, oracle_mod, dtype, with_gradp):
    case = inputs.cubes(shape=(64, 32, 24))
    h = wm.Handle.from_case(case, dtype=dtype)
    rng = np.random.default_rng(8)
    gp = [rounded(rng.standard_normal(case.shape), dtype) for _ in range(3)] if with_gradp else None
    u, v, w = (rounded(x, dtype) for x in (case.u, case.v, case.w))
    ud, vd, wd = (to_dev(x, dtype) for x in (u, v, w))
    dt = 0.0125
    h.mask(ud, vd, wd, None if gp is None else [to_dev(g, dtype) for g in gp], dt)
    uo, vo, wo = u.copy(), v.copy(), w.copy()
    oracle_mod.mask(case.grid, case.phi_uv, case.phi_w, uo, vo, wo, gp, dt)
    for got, ref in ((ud, uo), (vd, vo), (wd, wo)):
        g = to_host(got)
        if dtype == "f64":
            assert np.array_equal(g, ref)
        else:
            assert normwise(g, ref)[0] <= 2e-7


def test_degenerate_all_fluid_and_all_solid(wm, oracle_mod):
    for wall in (-0.5, 1.5):      # surface below the floor (no band) / above the lid (all solid)
        case = inputs.flat((16, 8, 9), wall_height=wall, sigma=0.3, seed=2, dtype="f32")
        h = wm.Handle.from_case(case, dtype="f32")
        assert h.list_size(wm.LIST_BAND_W) == 0 and h.list_size(wm.LIST_BAND_UV) == 0
        tau_g, f_g, st_g, _ = gpu_step(h, case, "f32")
        tau_o, f_o, st_o = oracle_step(oracle_mod, case)
        for k in inputs.TAU_NAMES:
            assert normwise(tau_g[k], tau_o[k])[0] <= TOL["f32"]
        for c in range(3):
            assert normwise(f_g[c], f_o[c])[0] <= TOL["f32"]
        assert st_g[0]["count"] == 0 and st_g[1]["count"] == 0
        assert st_g[0]["sum_tw"] == 0 and st_g[1]["max_ur"] == 0


def test_minimum_grid(wm, oracle_mod):
    case = inputs.flat((1, 1, 3), wall_height=0.4, sigma=0.3, seed=1, lengths=(0.1, 0.1, 1.0))
    for dtype in ("f32", "f64"):
        h = wm.Handle.from_case(case, dtype=dtype)
        tau_g, f_g, st_g, _ = gpu_step(h, case, dtype)
        tau_o, f_o, st_o = oracle_step(oracle_mod, case)
        for k in inputs.TAU_NAMES:
            assert normwise(tau_g[k], tau_o[k])[0] <= TOL[dtype]
        assert_stats_close(st_g, st_o, dtype)


def test_repeat_calls_deterministic_and_step_entry(wm):
    case = inputs.cubes(shape=(72, 40, 36))
    h = wm.Handle.from_case(case, dtype="f32")
    a = gpu_step(h, case, "f32")
    b = gpu_step(h, case, "f32")
    for k in inputs.TAU_NAMES:
        assert np.array_equal(a[0][k], b[0][k])
    for c in range(3):
        assert np.array_equal(a[1][c], b[1][c])
    assert a[2].tobytes() == b[2].tobytes()
    # the one-pass step entry point equals the three calls in order
    u, v, w = (to_dev(x, "f32") for x in (case.u, case.v, case.w))
    tau = [to_dev(case.tau[k], "f32") for k in inputs.TAU_NAMES]
    f = [to_dev(np.zeros(case.shape), "f32") for _ in range(3)]
    stats = h.new_stats()
    h.step(u, v, w, tau, f, None, 0.0, stats)
    torch.cuda.synchronize()
    for c in range(3):
        assert np.array_equal(to_host(f[c]), a[1][c])
    assert h.parse_stats(stats).tobytes() == a[2].tobytes()
    # the step masked the body velocity afterwards
    body = case.phi_uv <= 0
    assert np.all(to_host(u)[body] == 0)


def test_traffic_bytes(wm):
    case = inputs.cubes(shape=(64, 32, 24))
    for dtype, es in (("f32", 4), ("f64", 8)):
        h = wm.Handle.from_case(case, dtype=dtype)
        assert h.traffic_bytes(1) == 9 * es * case.npoints
        assert 0 < h.traffic_bytes(0) < h.traffic_bytes(1)
        assert h.traffic_bytes(3) > h.traffic_bytes(2) > 0


def test_binding_rejects_wrong_dtype(wm):
    case = inputs.ridge(shape=(16, 8, 8))
    h = wm.Handle.from_case(case, dtype="f32")
    bad = torch.zeros(case.shape, dtype=torch.float64, device="cuda")
    ok = torch.zeros(case.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        h.force([bad] * 6, [ok] * 3)


@pytest.mark.parametrize("name,dtype", [("cubes", "f32"), ("cubes", "f64"), ("hill", "f32")])
def test_full_size_parity(wm, oracle_mod, name, dtype):
    """Full-size workloads (4.2 M and 33.5 M nodes) in the launch configuration the
    benchmark times, against the full oracle."""
    case = inputs.make(name)
    h = wm.Handle.from_case(case, dtype=dtype)
    tau_g, f_g, st_g, _ = gpu_step(h, case, dtype)
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    for k in inputs.TAU_NAMES:
        assert normwise(tau_g[k], tau_o[k])[0] <= TOL[dtype], k
    for c in range(3):
        e, rms = normwise(f_g[c], f_o[c])
        print(name, dtype, "f" + "xyz"[c], "normwise", e, "rms", rms)
        assert e <= TOL[dtype]
    assert_stats_close(st_g, st_o, dtype)
    ref = oracle_lists(oracle_mod, case)
    for which in range(2):
        assert np.array_equal(h.export_list(which).astype(np.int64), ref[which])
