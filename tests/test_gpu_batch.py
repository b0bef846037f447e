"""Batched ensembles: members of uneven grid sizes stepped together give, member
by member, what single-terrain steps give, and match the FP64 oracle, in every
batch form: one cooperative launch with wall warps beside the stencil warps of
every block (force_path 6, the default) or with every member's band records as
interleaved wall stages of the stencil pipeline (force_path 5), and the batch
wall kernel followed by the batch stencil (force_path 3)."""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import TOL, assert_stats_close, normwise, oracle_step, poisoned_tau, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL_SHAPES = ((32, 16, 20), (48, 24, 16), (64, 32, 24), (40, 20, 18))


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


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_equals_single_steps_and_oracle(wm, oracle_mod, dtype):
    cases = [inputs.ensemble_member(m, shape=SMALL_SHAPES[m % len(SMALL_SHAPES)], dtype=dtype) for m in range(9)]
    handles = [wm.Handle.from_case(c, dtype=dtype) for c in cases]
    batch = wm.Batch(handles)
    fields = [_fields(c, dtype) for c in cases]
    batch.set_fields(fields)
    stats = batch.new_stats()
    batch.step(stats)
    torch.cuda.synchronize()
    bstats = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=wm.STATS_DTYPE).reshape(len(cases), 2)
    for m, (c, h) in enumerate(zip(cases, handles)):
        u, v, w, tau, f = _fields(c, dtype)
        st = h.new_stats()
        h.step(u, v, w, tau, f, None, 0.0, st)
        torch.cuda.synchronize()
        bu, bv, bw, btau, bf = fields[m]
        for got, ref in zip(bf, f):
            assert np.array_equal(to_host(got), to_host(ref)), m
        for got, ref in zip(btau, tau):
            assert np.array_equal(to_host(got), to_host(ref)), m
        for got, ref in zip((bu, bv, bw), (u, v, w)):
            assert np.array_equal(to_host(got), to_host(ref)), m
        tau_o, f_o, st_o = oracle_step(oracle_mod, c)
        for cc in range(3):
            assert normwise(to_host(bf[cc]), f_o[cc])[0] <= TOL[dtype], (m, cc)
        assert_stats_close(bstats[m], st_o, dtype)
    assert handles[0].device_status() == wm.OK
    batch.close()


def test_batch_graph_replay(wm):
    """The batch step captured once in a CUDA graph replays to the eager result."""
    cases = [inputs.ensemble_member(m, shape=SMALL_SHAPES[m % 4]) for m in range(6)]
    handles = [wm.Handle.from_case(c) for c in cases]
    batch = wm.Batch(handles)
    fields_a = [_fields(c, "f32") for c in cases]
    batch.set_fields(fields_a)
    batch.step()
    torch.cuda.synchronize()
    ref = [[to_host(t) for t in fa[4]] for fa in fields_a]
    fields_b = [_fields(c, "f32") for c in cases]
    batch.set_fields(fields_b)
    stats = batch.new_stats()
    batch.step(stats)        # warm up outside the capture
    torch.cuda.synchronize()
    for fb, c in zip(fields_b, cases):      # reset the inputs the step modified
        fb[0].copy_(to_dev(c.u, "f32")); fb[1].copy_(to_dev(c.v, "f32")); fb[2].copy_(to_dev(c.w, "f32"))
        for t, k in zip(fb[3], inputs.TAU_NAMES):
            t.copy_(to_dev(c.tau[k], "f32"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.step(stats)
    for fb, c in zip(fields_b, cases):
        fb[0].copy_(to_dev(c.u, "f32")); fb[1].copy_(to_dev(c.v, "f32")); fb[2].copy_(to_dev(c.w, "f32"))
        for t, k in zip(fb[3], inputs.TAU_NAMES):
            t.copy_(to_dev(c.tau[k], "f32"))
    g.replay()
    torch.cuda.synchronize()
    for m, fb in enumerate(fields_b):
        for got, r in zip(fb[4], ref[m]):
            assert np.array_equal(to_host(got), r), m
    batch.close()


BATCH_TUNINGS = [dict(rows=1, stages=3, consumer_warps=2), dict(rows=2, stages=5, consumer_warps=8),
                 dict(rows=4, stages=2, consumer_warps=4, blocks_per_sm=1),
                 dict(rows=2, stages=4, consumer_warps=6, wall_chunk=64),
                 dict(rows=4, stages=3, consumer_warps=3, wall_chunk=2048),
                 dict(rows=1, stages=6, consumer_warps=4, wall_chunk=200),
                 dict(rows=2, stages=3, consumer_warps=3, wall_warps=2),
                 dict(rows=4, stages=2, consumer_warps=5, wall_warps=6),
                 dict(rows=4, stages=3, consumer_warps=4, wall_warps=3, dyn_chunk=1),
                 dict(rows=2, stages=3, consumer_warps=3, wall_warps=2, dyn_chunk=13)]


@pytest.mark.parametrize("form", [3, 5, 6])
@pytest.mark.parametrize("tuning", range(len(BATCH_TUNINGS)))
def test_batch_tunings(wm, oracle_mod, tuning, form):
    """Every batch form and a covering set of tile shapes and band-record chunks,
    against the oracle: stresses, forcing and statistics, with the outputs NaN
    before the call."""
    cases = [inputs.ensemble_member(m, shape=SMALL_SHAPES[m % 4]) for m in range(5)]
    handles = [wm.Handle.from_case(c) for c in cases]
    batch = wm.Batch(handles)
    tun = dict(BATCH_TUNINGS[tuning], force_path=form)
    batch.set_tuning(**tun)
    fields = [_fields(c, "f32") for c in cases]
    for fl in fields:
        for t in fl[4]:
            t.fill_(float("nan"))
    batch.set_fields(fields)
    stats = batch.new_stats()
    batch.wall_stress_force(stats)
    torch.cuda.synchronize()
    bstats = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=wm.STATS_DTYPE).reshape(len(cases), 2)
    for m, c in enumerate(cases):
        tau_o, f_o, st_o = oracle_step(oracle_mod, c)
        for k, t in zip(inputs.TAU_NAMES, fields[m][3]):
            assert normwise(to_host(t), tau_o[k])[0] <= TOL["f32"], (tun, m, k)
        for cc in range(3):
            g = to_host(fields[m][4][cc])
            assert np.all(np.isfinite(g)), (tun, m, cc)
            assert normwise(g, f_o[cc])[0] <= TOL["f32"], (tun, m)
        assert_stats_close(bstats[m], st_o, "f32")
    assert handles[0].device_status() == wm.OK
    batch.close()


@pytest.mark.parametrize("form", [3, 5, 6])
def test_batch_forms_bitwise_equal_and_replay(wm, form):
    """Both batch forms give the same stresses and forcing bit for bit (the same
    per-node arithmetic), from a CUDA graph replayed twice."""
    cases = [inputs.ensemble_member(m, shape=SMALL_SHAPES[m % 4]) for m in range(6)]
    handles = [wm.Handle.from_case(c) for c in cases]
    batch = wm.Batch(handles)
    batch.set_tuning(force_path=3)
    ref = [_fields(c, "f32") for c in cases]
    batch.set_fields(ref)
    batch.wall_stress_force()
    torch.cuda.synchronize()
    batch.set_tuning(force_path=form)
    fields = [_fields(c, "f32") for c in cases]
    batch.set_fields(fields)
    stats = batch.new_stats()
    batch.wall_stress_force(stats)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.wall_stress_force(stats)
    for _ in range(2):
        for fl in fields:
            for t in fl[4]:
                t.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for m in range(len(cases)):
            for got, r in zip(fields[m][3] + fields[m][4], ref[m][3] + ref[m][4]):
                assert np.array_equal(to_host(got), to_host(r)), (form, m)
    assert handles[0].device_status() == wm.OK
    batch.close()


def test_full_ensemble_64(wm, oracle_mod):
    """The 64-member ensemble (grids 64^3 .. 256x128x64) in both batch forms, every
    member's stresses, forcing and statistics against the oracle."""
    cases = inputs.ensemble(64)
    handles = [wm.Handle.from_case(c) for c in cases]
    batch = wm.Batch(handles)
    out = {}
    for form in (6, 5, 3):
        batch.set_tuning(force_path=form)
        fields = [_fields(c, "f32") for c in cases]
        batch.set_fields(fields)
        stats = batch.new_stats()
        batch.wall_stress_force(stats)
        torch.cuda.synchronize()
        out[form] = (fields, np.frombuffer(stats.cpu().numpy().tobytes(), dtype=wm.STATS_DTYPE).reshape(64, 2))
    for m, c in enumerate(cases):
        tau_o, f_o, st_o = oracle_step(oracle_mod, c)
        for form, (fields, bstats) in out.items():
            for k, t in zip(inputs.TAU_NAMES, fields[m][3]):
                assert normwise(to_host(t), tau_o[k])[0] <= TOL["f32"], (form, m, k)
            for cc in range(3):
                assert normwise(to_host(fields[m][4][cc]), f_o[cc])[0] <= TOL["f32"], (form, m, cc)
            assert_stats_close(bstats[m], st_o, "f32")
    assert batch.points() == sum(c.npoints for c in cases)
    assert handles[0].device_status() == wm.OK
    batch.close()


def test_batch_wall_stress_force_equals_single_calls(wm):
    """The batch step without the mask: stresses and forcing equal the single-terrain
    wall_stress_force of every member, and the velocity is left untouched."""
    cases = [inputs.ensemble_member(m, shape=SMALL_SHAPES[m % len(SMALL_SHAPES)]) for m in range(7)]
    handles = [wm.Handle.from_case(c) for c in cases]
    batch = wm.Batch(handles)
    fields = [_fields(c, "f32") for c in cases]
    batch.set_fields(fields)
    stats = batch.new_stats()
    batch.wall_stress_force(stats)
    torch.cuda.synchronize()
    bstats = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=wm.STATS_DTYPE).reshape(len(cases), 2)
    for m, (c, h) in enumerate(zip(cases, handles)):
        u, v, w, tau, f = _fields(c, "f32")
        st = h.new_stats()
        h.wall_stress_force(u, v, w, tau, f, st)
        torch.cuda.synchronize()
        bu, bv, bw, btau, bf = fields[m]
        for got, ref in zip(btau + bf, tau + f):
            assert np.array_equal(to_host(got), to_host(ref)), m
        for got, src in zip((bu, bv, bw), (c.u, c.v, c.w)):
            assert np.array_equal(to_host(got), to_host(to_dev(src, "f32"))), m
        single = h.parse_stats(st)
        for bnd in range(2):
            assert bstats[m][bnd]["count"] == single[bnd]["count"]
            assert bstats[m][bnd]["sum_tw"] == pytest.approx(single[bnd]["sum_tw"], rel=1e-5)
    batch.close()


@pytest.mark.parametrize("form", [3, 5, 6])
def test_batch_of_one(wm, oracle_mod, form):
    """A batch of a single member (its launch reads the member from the kernel
    parameters, not from the descriptor array) matches the oracle."""
    case = inputs.ensemble_member(3, shape=(64, 32, 24))
    h = wm.Handle.from_case(case)
    batch = wm.Batch([h])
    batch.set_tuning(force_path=form)
    fields = [_fields(case, "f32")]
    batch.set_fields(fields)
    stats = batch.new_stats()
    batch.wall_stress_force(stats)
    torch.cuda.synchronize()
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    for k, t in zip(inputs.TAU_NAMES, fields[0][3]):
        assert normwise(to_host(t), tau_o[k])[0] <= TOL["f32"], k
    for cc in range(3):
        assert normwise(to_host(fields[0][4][cc]), f_o[cc])[0] <= TOL["f32"], cc
    bstats = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=wm.STATS_DTYPE).reshape(1, 2)
    assert_stats_close(bstats[0], st_o, "f32")
    batch.close()


def _empty_member(seed):
    """A member whose wall lies below the floor: no band node, no solid node."""
    return inputs.flat((24, 16, 10), wall_height=-1.0, lengths=(1.0, 1.0, 1.0), sigma=0.2, seed=seed, dtype="f32")


@pytest.mark.parametrize("form", [3, 5, 6])
@pytest.mark.parametrize("layout", ["mixed", "all_empty"])
def test_batch_with_empty_members(wm, oracle_mod, form, layout):
    """Members without band records or solid runs, between members with both (their
    record and run offsets repeat in the member table) or making up the whole batch
    (no record and no run at all), leave the fluid stress as it is, report empty
    statistics, and do not disturb the others: every member matches the oracle."""
    if layout == "mixed":
        cases = [_empty_member(11), inputs.ensemble_member(1, shape=(48, 24, 16)), _empty_member(12),
                 _empty_member(13), inputs.flat((40, 20, 12), wall_height=0.3, sigma=0.2, seed=14, dtype="f32"),
                 inputs.ensemble_member(2, shape=(32, 16, 20)), _empty_member(15)]
    else:
        cases = [_empty_member(21), _empty_member(22), _empty_member(23)]
    handles = [wm.Handle.from_case(c) for c in cases]
    batch = wm.Batch(handles)
    batch.set_tuning(force_path=form)
    fields = []
    for c in cases:                       # NaN where the wall model writes, so that a skipped entry shows up
        u, v, w, _, f = _fields(c, "f32")
        pt = poisoned_tau(c)
        fields.append((u, v, w, [to_dev(pt[k], "f32") for k in inputs.TAU_NAMES], f))
    batch.set_fields(fields)
    stats = batch.new_stats()
    for _ in range(2):                    # the second call finds the counters and scratch re-armed
        batch.wall_stress_force(stats)
    torch.cuda.synchronize()
    assert batch.device_status() == wm.OK
    bstats = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=wm.STATS_DTYPE).reshape(len(cases), 2)
    for m, c in enumerate(cases):
        tau_o, f_o, st_o = oracle_step(oracle_mod, c)
        for k, t in zip(inputs.TAU_NAMES, fields[m][3]):
            got = to_host(t)
            assert np.all(np.isfinite(got)), (m, k)
            assert normwise(got, tau_o[k])[0] <= TOL["f32"], (m, k)
        for cc in range(3):
            assert normwise(to_host(fields[m][4][cc]), f_o[cc])[0] <= TOL["f32"], (m, cc)
        assert_stats_close(bstats[m], st_o, "f32")
        if float(np.min(c.phi_w)) >= 1.0:          # the members with the wall below the floor
            for k, t in zip(inputs.TAU_NAMES, fields[m][3]):
                assert np.array_equal(to_host(t), c.tau[k].astype(np.float32)), (m, k)
            assert bstats[m][0]["count"] == 0 and bstats[m][1]["count"] == 0
    batch.close()
