"""GPU parity of the CUDA stress stage against the FP64 oracle, through the C ABI.

Tolerances (normwise, max |gpu - oracle| / max |oracle| per array): 1e-12 for
the FP64 path and 1e-5 for the FP32 path; index lists are compared bit-exactly;
band statistics to 1e-11 (FP64) / 1e-5 (FP32) relative.
"""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import (TOL, assert_stats_close, gpu_fused, gpu_step, normwise, oracle_lists, oracle_step,
                         rounded, to_dev, to_host)

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
    # the step takes the fused pass: same values up to rounding, statistics summed
    # in another order
    for c in range(3):
        assert normwise(to_host(f[c]), a[1][c])[0] <= 1e-6
    st = h.parse_stats(stats)
    for bnd in range(2):
        assert st[bnd]["count"] == a[2][bnd]["count"]
        assert st[bnd]["sum_tw"] == pytest.approx(a[2][bnd]["sum_tw"], rel=1e-5)
        assert st[bnd]["max_ur"] == pytest.approx(a[2][bnd]["max_ur"], rel=1e-6)
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


@pytest.mark.parametrize("dtype,es", [("f32", 4), ("f64", 8)])
def test_sector_traffic(wm, dtype, es):
    """The wall stage's bytes at 32-byte sector granularity: the written stress
    sectors recounted from the exported band and solid lists; the sector reads hold
    each written sector once plus the element-level reads rounded up to sectors."""
    case = inputs.cubes(shape=(64, 32, 24))
    h = wm.Handle.from_case(case, dtype=dtype)
    per = 32 // es
    n = case.npoints
    written = 0
    for comps, lists in ((2, (wm.LIST_BAND_W, wm.LIST_SOLID_W)), (4, (wm.LIST_BAND_UV, wm.LIST_SOLID_UV))):
        mask = np.zeros(n + (-n) % per, bool)
        for l in lists:
            mask[h.export_list(l)] = True
        written += comps * int(mask.reshape(-1, per).any(axis=1).sum())
    assert h.traffic_bytes(6) == 32 * written
    element_reads = h.traffic_bytes(0) - es * sum(
        c * h.list_size(l) for c, l in ((2, wm.LIST_BAND_W), (4, wm.LIST_BAND_UV), (2, wm.LIST_SOLID_W),
                                        (4, wm.LIST_SOLID_UV)))
    # records and run descriptors are in both counts; velocity elements round up to their sectors
    rest = h.traffic_bytes(5) - h.traffic_bytes(6)
    assert element_reads <= rest <= per * element_reads
    h.close()


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


def _check_against_oracle(tau_g, f_g, st_g, tau_o, f_o, st_o, dtype, label):
    for k in inputs.TAU_NAMES:
        e, _ = normwise(tau_g[k], tau_o[k])
        assert e <= TOL[dtype], (label, k, e)
    for c in range(3):
        e, _ = normwise(f_g[c], f_o[c])
        assert e <= TOL[dtype], (label, "f" + "xyz"[c], e)
    if st_g is not None:
        assert_stats_close(st_g, st_o, dtype)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_pass_parity(wm, oracle_mod, name, dtype):
    """One fused pass (pipelined stencil with the band wall model applied to the
    staged rows) against the oracle's wall stress followed by its force."""
    case = CASES[name]()
    h = wm.Handle.from_case(case, dtype=dtype)
    tau_g, f_g, st_g = gpu_fused(h, case, dtype)
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    _check_against_oracle(tau_g, f_g, st_g, tau_o, f_o, st_o, dtype, name)
    assert h.device_status() == wm.OK


TUNINGS = [
    dict(rows=1, stages=2, consumer_warps=1, wall_warps=1),
    dict(rows=2, stages=3, consumer_warps=4, wall_warps=2),
    dict(rows=4, stages=2, consumer_warps=8, wall_warps=4),
    dict(rows=2, stages=6, consumer_warps=2, wall_warps=1, blocks_per_sm=1),
    dict(rows=1, stages=4, consumer_warps=12, wall_warps=3),
    dict(force_path=2, direct_bx=16, direct_by=4, direct_kc=8),
    dict(force_path=2, direct_bx=8, direct_by=2, direct_kc=1),
]


@pytest.mark.parametrize("tuning", range(len(TUNINGS)))
@pytest.mark.parametrize("name", ["cubes_small", "hill_even"])
def test_tunings_give_the_same_answer(wm, oracle_mod, tuning, name):
    """Every launch shape the autotuner may pick keeps parity (fused and separate)."""
    case = inputs.cubes(shape=(72, 40, 36)) if name == "cubes_small" else inputs.hill(shape=(96, 48, 40))
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    for dtype in ("f32", "f64"):
        h = wm.Handle.from_case(case, dtype=dtype)
        h.set_tuning(**TUNINGS[tuning])
        tau_g, f_g, st_g = gpu_fused(h, case, dtype)
        _check_against_oracle(tau_g, f_g, st_g, tau_o, f_o, st_o, dtype, (name, tuning, "fused"))
        tau_g, f_g, st_g, _ = gpu_step(h, case, dtype)
        _check_against_oracle(tau_g, f_g, st_g, tau_o, f_o, st_o, dtype, (name, tuning, "separate"))
        assert h.device_status() == wm.OK


def test_fused_equals_separate_calls(wm):
    case = inputs.hill(shape=(128, 64, 48))
    h = wm.Handle.from_case(case, dtype="f32")
    a = gpu_fused(h, case, "f32")
    b = gpu_step(h, case, "f32")
    for k in inputs.TAU_NAMES:
        assert normwise(a[0][k], b[0][k])[0] <= 1e-6
    for c in range(3):
        assert normwise(a[1][c], b[1][c])[0] <= 1e-6
    for bnd in range(2):
        assert a[2][bnd]["count"] == b[2][bnd]["count"]
        assert a[2][bnd]["min_tw"] == pytest.approx(b[2][bnd]["min_tw"], rel=1e-6)
        assert a[2][bnd]["sum_tw"] == pytest.approx(b[2][bnd]["sum_tw"], rel=1e-5)


def test_set_tuning_rejects_bad_fields(wm):
    case = inputs.ridge(shape=(16, 8, 8))
    h = wm.Handle.from_case(case, dtype="f32")
    for bad in (dict(rows=3), dict(stages=9), dict(consumer_warps=13), dict(force_path=7), dict(wall_chunk=-1),
                dict(wall_chunk=65537), dict(dyn_chunk=-1), dict(dyn_chunk=4097)):
        with pytest.raises(wm.WmibmError):
            h.set_tuning(**bad)


@pytest.mark.parametrize("name,dtype", [("cubes", "f32"), ("hill", "f32"), ("cubes", "f64")])
def test_full_size_fused_parity(wm, oracle_mod, name, dtype):
    """The fused pass the benchmark times, at full size, against the full oracle."""
    case = inputs.make(name)
    h = wm.Handle.from_case(case, dtype=dtype)
    tau_g, f_g, st_g = gpu_fused(h, case, dtype)
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    _check_against_oracle(tau_g, f_g, st_g, tau_o, f_o, st_o, dtype, name)
    assert h.device_status() == wm.OK


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("with_gradp", [False, True])
def test_force_mask_equals_force_then_mask(wm, oracle_mod, dtype, with_gradp):
    """The one-launch force + mask against the oracle's force and Eq. 27 mask."""
    case = inputs.hill(shape=(96, 48, 40))
    h = wm.Handle.from_case(case, dtype=dtype)
    rng = np.random.default_rng(12)
    tau = {k: rounded(rng.standard_normal(case.shape), dtype) for k in inputs.TAU_NAMES}
    gp = [rounded(rng.standard_normal(case.shape), dtype) for _ in range(3)] if with_gradp else None
    u, v, w = (rounded(x, dtype) for x in (case.u, case.v, case.w))
    td = [to_dev(tau[k], dtype) for k in inputs.TAU_NAMES]
    f = [to_dev(np.zeros(case.shape), dtype) for _ in range(3)]
    ud, vd, wd = (to_dev(x, dtype) for x in (u, v, w))
    dt = 0.02
    h.force_mask(td, f, ud, vd, wd, None if gp is None else [to_dev(g, dtype) for g in gp], dt)
    ref_f = oracle_mod.force(case.grid, tau)
    uo, vo, wo = u.copy(), v.copy(), w.copy()
    oracle_mod.mask(case.grid, case.phi_uv, case.phi_w, uo, vo, wo, gp, dt)
    for c in range(3):
        assert normwise(to_host(f[c]), ref_f[c])[0] <= (1e-14 if dtype == "f64" else 2e-7)
    for got, ref in ((ud, uo), (vd, vo), (wd, wo)):
        assert normwise(to_host(got), ref)[0] <= (0.0 if dtype == "f64" else 2e-7)
    assert h.device_status() == wm.OK


def test_step_full_pass_against_oracle(wm, oracle_mod):
    """wmibm_step (wall kernel, then force + mask in one launch) against the
    oracle's wall stress, force and mask in that order."""
    case = inputs.cubes(shape=(128, 64, 48))
    h = wm.Handle.from_case(case, dtype="f32")
    u, v, w = (to_dev(x, "f32") for x in (case.u, case.v, case.w))
    tau = [to_dev(case.tau[k], "f32") for k in inputs.TAU_NAMES]
    f = [to_dev(np.zeros(case.shape), "f32") for _ in range(3)]
    stats = h.new_stats()
    h.step(u, v, w, tau, f, None, 0.0, stats)
    torch.cuda.synchronize()
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    uo, vo, wo = case.u.copy(), case.v.copy(), case.w.copy()
    oracle_mod.mask(case.grid, case.phi_uv, case.phi_w, uo, vo, wo)
    for c in range(3):
        assert normwise(to_host(f[c]), f_o[c])[0] <= TOL["f32"]
    for k, t in zip(inputs.TAU_NAMES, tau):
        assert normwise(to_host(t), tau_o[k])[0] <= TOL["f32"]
    for got, ref in ((u, uo), (v, vo), (w, wo)):
        assert normwise(to_host(got), ref)[0] <= TOL["f32"]
    assert_stats_close(h.parse_stats(stats), st_o, "f32")
    assert h.device_status() == wm.OK
