"""Every launch form and a covering set of the tile shapes the autotuner may pick,
against the FP64 oracle, on a full-width slab of the cube array (256 x 128 x 40).

The autotuner times these shapes and keeps the fastest, so the shape behind a
benchmark number is one of them.  The forms are the single cooperative launch
with the wall model in every block (force_path 1), the direct-load force
kernel (2), the wall kernel followed by the pipelined stencil (3), dedicated
wall blocks (4), the band records as interleaved pipeline stages (5) and wall
warps beside the producer and consumers of every block (6).  The
covering set gives each value of every field (rows per strip, stages, consumer
warps, warps of the wall kernel, records per wall stage, units per take of the
dynamic dispensing) at least once per form.
The forcing and stress outputs start as NaN where the stage writes them, so a
skipped write shows up; tolerances are those of the parity tests (Sec. 3.3 wall
model, Eq. 18 forcing).
"""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import TOL, assert_stats_close, normwise, oracle_step, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SLAB = (256, 128, 40)

# (rows, stages, consumer_warps, wall_warps, wall_chunk[, dyn_chunk]) per force_path
SHAPES = {
    1: [(1, 2, 2, 0, 0), (2, 3, 4, 0, 0), (4, 4, 8, 0, 0), (2, 6, 3, 0, 0), (1, 5, 6, 0, 0), (4, 3, 2, 0, 0)],
    3: [(1, 2, 2, 4, 0), (2, 3, 4, 8, 0), (4, 3, 8, 8, 0), (2, 6, 3, 4, 0), (1, 5, 6, 8, 0), (4, 2, 2, 4, 0),
        (2, 3, 4, 8, 0, 1), (4, 3, 4, 8, 0, 7), (1, 2, 3, 4, 0, 64)],
    4: [(1, 3, 2, 0, 0), (2, 4, 4, 0, 0), (4, 3, 8, 0, 0), (2, 6, 6, 0, 0), (1, 2, 3, 0, 0)],
    5: [(1, 2, 2, 0, 0), (2, 3, 4, 0, 64), (4, 3, 8, 0, 512), (2, 6, 3, 0, 1024), (1, 5, 6, 0, 256),
        (4, 2, 4, 0, 4096)],
    6: [(1, 2, 2, 1, 0), (2, 3, 4, 3, 0), (4, 3, 8, 4, 0), (2, 6, 3, 2, 0), (1, 5, 6, 8, 0), (4, 2, 4, 6, 0),
        (4, 3, 4, 3, 0, 1), (2, 3, 3, 2, 0, 5), (4, 2, 4, 3, 0, 16), (1, 4, 4, 4, 0, 4096)],
    2: [(0, 0, 0, 0, 0)],
}
CASES = [(fp, i) for fp in sorted(SHAPES) for i in range(len(SHAPES[fp]))]


@pytest.fixture(scope="module")
def wm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03343_gb300 import build, wmibm
    build.build()
    wmibm.load()
    return wmibm


@pytest.fixture(scope="module")
def slab_ref(oracle_mod):
    case = inputs.cubes(shape=SLAB)
    return case, oracle_step(oracle_mod, case)


def _tuning(fp, shape):
    rows, stages, cons, wall, chunk = shape[:5]
    dyn = shape[5] if len(shape) > 5 else 0
    t = dict(force_path=fp)
    for k, v in (("rows", rows), ("stages", stages), ("consumer_warps", cons), ("wall_warps", wall),
                 ("wall_chunk", chunk), ("dyn_chunk", dyn)):
        if v:
            t[k] = v
    return t


def _poisoned_fields(case, dtype):
    """Velocity and stresses from the case; the forcing all NaN, and the stress NaN at
    every band and solid node (the entries the wall model writes)."""
    u, v, w = (to_dev(x, dtype) for x in (case.u, case.v, case.w))
    tau = []
    for k in inputs.TAU_NAMES:
        a = case.tau[k].copy()
        phi = case.phi_w if inputs.TAU_ON_W[k] else case.phi_uv
        lim = case.phi_b if inputs.TAU_ON_W[k] else 2.0 * case.phi_b
        a[phi <= lim] = np.nan
        tau.append(to_dev(a, dtype))
    f = [to_dev(np.full(case.shape, np.nan), dtype) for _ in range(3)]
    return u, v, w, tau, f


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("fp,i", CASES)
def test_shape_against_oracle(wm, slab_ref, fp, i, dtype):
    case, (tau_o, f_o, st_o) = slab_ref
    tuning = _tuning(fp, SHAPES[fp][i])
    h = wm.Handle.from_case(case, dtype=dtype)
    try:
        h.set_tuning(**tuning)
    except wm.WmibmError:
        pytest.skip(f"{tuning} is not a valid shape here")
    u, v, w, tau, f = _poisoned_fields(case, dtype)
    st = h.new_stats()
    try:
        h.wall_stress_force(u, v, w, tau, f, st)
    except wm.WmibmError as e:
        if e.status == wm.EINVAL:       # a shape that does not fit the shared memory of this precision
            pytest.skip(str(e))
        raise
    torch.cuda.synchronize()
    for k, t in zip(inputs.TAU_NAMES, tau):
        g = to_host(t)
        assert np.all(np.isfinite(g)), (tuning, k)
        e, _ = normwise(g, tau_o[k])
        assert e <= TOL[dtype], (tuning, k, e)
    for c in range(3):
        g = to_host(f[c])
        assert np.all(np.isfinite(g)), (tuning, c)
        e, _ = normwise(g, f_o[c])
        assert e <= TOL[dtype], (tuning, "f" + "xyz"[c], e)
    assert_stats_close(h.parse_stats(st), st_o, dtype)
    assert h.device_status() == wm.OK
    h.close()


@pytest.mark.parametrize("fp", [1, 3, 4, 5, 6])
def test_shape_graph_replay_and_step(wm, oracle_mod, fp):
    """One shape per form captured in a CUDA graph and replayed twice (the launch
    re-arms its counters), then the whole step with the body mask (Eq. 27)."""
    case = inputs.cubes(shape=(128, 64, 48))
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    h = wm.Handle.from_case(case, dtype="f32")
    h.set_tuning(**_tuning(fp, SHAPES[fp][1]))
    u, v, w, tau, f = _poisoned_fields(case, "f32")
    st = h.new_stats()
    call = h.prepare_step(u, v, w, tau, f, st)
    call.wall_stress_force()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        call.wall_stress_force()
    for _ in range(2):
        for t in f:
            t.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for c in range(3):
            assert normwise(to_host(f[c]), f_o[c])[0] <= TOL["f32"], (fp, c)
        assert_stats_close(h.parse_stats(st), st_o, "f32")
    # the step with the mask, from fresh fields
    u, v, w, tau, f = _poisoned_fields(case, "f32")
    h.step(u, v, w, tau, f, None, 0.0, st)
    torch.cuda.synchronize()
    uo, vo, wo = case.u.copy(), case.v.copy(), case.w.copy()
    oracle_mod.mask(case.grid, case.phi_uv, case.phi_w, uo, vo, wo)
    for got, ref in ((u, uo), (v, vo), (w, wo)):
        assert normwise(to_host(got), ref)[0] <= TOL["f32"]
    for c in range(3):
        assert normwise(to_host(f[c]), f_o[c])[0] <= TOL["f32"]
    assert h.device_status() == wm.OK
    h.close()


def test_autotuner_keeps_a_shape_that_agrees(wm, oracle_mod):
    """The autotuner's pick (from a short sweep) agrees with the default shape and
    with the oracle."""
    from paper_2006_03343_gb300 import autotune
    case = inputs.cubes(shape=(128, 64, 40))
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    h = wm.Handle.from_case(case, dtype="f32")
    u, v, w, tau, f = _poisoned_fields(case, "f32")
    st = h.new_stats()
    res = autotune.tune(h, (u, v, w, tau, f, st), reps=3, use_cache=False, budget_s=8.0)
    assert res["tuning"] and res["agreement"] <= autotune.AGREE["f32"]
    assert h.get_tuning().force_path == res["tuning"]["force_path"]
    u, v, w, tau, f = _poisoned_fields(case, "f32")
    h.wall_stress_force(u, v, w, tau, f, st)
    torch.cuda.synchronize()
    for c in range(3):
        assert normwise(to_host(f[c]), f_o[c])[0] <= TOL["f32"]
    assert_stats_close(h.parse_stats(st), st_o, "f32")
    h.close()


def test_batch_autotuner_keeps_a_shape_that_agrees(wm, oracle_mod):
    from paper_2006_03343_gb300 import autotune
    cases = [inputs.ensemble_member(m, shape=((64, 32, 24), (96, 48, 32), (128, 64, 24))[m % 3]) for m in range(5)]
    handles = [wm.Handle.from_case(c) for c in cases]
    batch = wm.Batch(handles)
    fields = [_poisoned_fields(c, "f32") for c in cases]
    batch.set_fields(fields)
    stats = batch.new_stats()
    res = autotune.tune_batch(batch, stats, reps=3, use_cache=False, budget_s=10.0)
    assert res["tuning"] and res["agreement"] <= autotune.AGREE["f32"]
    assert set(res["forms_ms"]) <= {"interleaved", "two_launch", "wall_warps"}
    for fl in fields:
        for t in fl[4]:
            t.fill_(float("nan"))
    batch.wall_stress_force(stats)
    torch.cuda.synchronize()
    for m, c in enumerate(cases):
        tau_o, f_o, _ = oracle_step(oracle_mod, c)
        for cc in range(3):
            assert normwise(to_host(fields[m][4][cc]), f_o[cc])[0] <= TOL["f32"], (m, cc)
    batch.close()
