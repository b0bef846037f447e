"""The single-launch stage (wall phase inside the cooperative stencil launch):
identical stresses, forcing and masked velocity to the two-launch form
(tuning.force_path = 3), statistics within tolerance, repeatable from a CUDA
graph (the launch re-arms its counters), and correct where the grid is capped
by the statistics scratch."""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import STATS_TOL, TOL, assert_stats_close, normwise, oracle_step, to_dev, to_host

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


def _fields(case, dtype):
    u, v, w = (to_dev(x, dtype) for x in (case.u, case.v, case.w))
    tau = [to_dev(case.tau[k], dtype) for k in inputs.TAU_NAMES]
    f = [to_dev(np.zeros(case.shape), dtype) for _ in range(3)]
    return u, v, w, tau, f


def _run(h, case, dtype, entry, gradp=None, dt=0.0):
    u, v, w, tau, f = _fields(case, dtype)
    st = h.new_stats()
    if entry == "step":
        h.step(u, v, w, tau, f, gradp, dt, st)
    else:
        h.wall_stress_force(u, v, w, tau, f, st)
    torch.cuda.synchronize()
    return [to_host(t) for t in tau], [to_host(t) for t in f], [to_host(t) for t in (u, v, w)], h.parse_stats(st)


TUNINGS = [dict(), dict(rows=1, stages=6, consumer_warps=2), dict(rows=4, stages=3, consumer_warps=8),
           dict(rows=2, stages=2, consumer_warps=1)]


@pytest.mark.parametrize("form", [1, 4])        # wall share in every block / dedicated wall blocks
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("entry", ["step", "wall_stress_force"])
@pytest.mark.parametrize("tuning", range(len(TUNINGS)))
def test_single_launch_equals_two_launches(wm, dtype, entry, tuning, form):
    case = inputs.cubes(shape=(96, 48, 40))
    h = wm.Handle.from_case(case, dtype=dtype)
    gp = None
    dt = 0.0
    if entry == "step":
        rng = np.random.default_rng(4)
        gp = [to_dev(rng.standard_normal(case.shape), dtype) for _ in range(3)]
        dt = 0.01
    h.set_tuning(force_path=form, **TUNINGS[tuning])
    one = _run(h, case, dtype, entry, gp, dt)
    h.set_tuning(force_path=3, **TUNINGS[tuning])
    two = _run(h, case, dtype, entry, gp, dt)
    for a, b in zip(one[0] + one[1] + one[2], two[0] + two[1] + two[2]):
        assert np.array_equal(a, b)
    for bnd in range(2):
        assert one[3][bnd]["count"] == two[3][bnd]["count"]
        for k in ("sum_tw", "sum_tw2", "min_tw", "max_ur"):
            ref = two[3][bnd][k]
            assert abs(one[3][bnd][k] - ref) <= STATS_TOL[dtype] * max(abs(ref), 1e-30)
    assert h.device_status() == wm.OK


@pytest.mark.parametrize("form", [1, 4])
def test_single_launch_graph_replays(wm, form):
    """Captured once, replayed many times: every replay gives the eager result."""
    case = inputs.cubes(shape=(128, 64, 48))
    h = wm.Handle.from_case(case, dtype="f32")
    h.set_tuning(force_path=form)
    ref = _run(h, case, "f32", "wall_stress_force")
    u, v, w, tau, f = _fields(case, "f32")
    st = h.new_stats()
    call = h.prepare_step(u, v, w, tau, f, st)
    call.wall_stress_force()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        call.wall_stress_force()
    for _ in range(6):
        for t, src in zip(tau, case.tau.values()):
            t.copy_(torch.from_numpy(np.ascontiguousarray(src)).to(t.dtype))
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip([to_host(t) for t in tau] + [to_host(t) for t in f], ref[0] + ref[1]):
            assert np.array_equal(a, b)
        stats = h.parse_stats(st)
        for bnd in range(2):
            assert stats[bnd]["count"] == ref[3][bnd]["count"]
            assert stats[bnd]["sum_tw"] == pytest.approx(ref[3][bnd]["sum_tw"], rel=1e-5)
    assert h.device_status() == wm.OK


@pytest.mark.parametrize("form", [1, 4])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_many_small_blocks_against_oracle(wm, oracle_mod, dtype, form):
    """One consumer warp per block on a small grid: the occupancy-sized grid is
    larger than the statistics scratch and is capped; results still match the oracle."""
    case = inputs.ridge(shape=(32, 32, 32), dtype=dtype)
    h = wm.Handle.from_case(case, dtype=dtype)
    h.set_tuning(force_path=form, rows=1, stages=2, consumer_warps=1)
    tau_g, f_g, _, st_g = _run(h, case, dtype, "wall_stress_force")
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    for c in range(3):
        assert normwise(f_g[c], f_o[c])[0] <= TOL[dtype]
    for k, t in zip(inputs.TAU_NAMES, tau_g):
        assert normwise(t, tau_o[k])[0] <= TOL[dtype]
    assert_stats_close(st_g, st_o, dtype)
    assert h.device_status() == wm.OK


def test_single_launch_with_log_z0(wm, oracle_mod):
    """The single launch honours the per-cell ln z0 field."""
    case, _ = inputs.adjoint_case(shape=(64, 32, 24), dtype="f64")
    s = np.log(case.z0)
    h = wm.Handle.from_case(case, dtype="f64")
    sd = to_dev(s, "f64")
    h.set_log_z0(sd)
    tau_g, f_g, _, _ = _run(h, case, "f64", "wall_stress_force")
    tau_o = {k: t.copy() for k, t in case.tau.items()}
    oracle_mod.wall_stress(case.grid, case.phi_uv, case.phi_w, None, case.phi_c, case.phi_b, case.u, case.v,
                           case.w, tau_o, logz0=s)
    f_o = oracle_mod.force(case.grid, tau_o)
    for c in range(3):
        assert normwise(f_g[c], f_o[c])[0] <= TOL["f64"]
