"""GPU Smagorinsky stress with Mason's wall damping (wmibm_sgs_wall_terms,
wmibm_sgs_stress, and the fused wmibm_sgs_force: Eqs. 4-7) against the FP64
oracle's sgs_stress on the same seeded inputs: every stress array element by
element (fluid entries written, all others kept) on small and ragged grids in
FP32 and FP64, per-cell z0, BF16 velocity storage, the minimal 3-level grid and
the full 256 x 128 x 128 cubes grid; the stage SGS -> wall stress -> forcing
against the oracle's chain, unfused and fused; the node markers; graph replay;
and argument checks."""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import TOL, normwise, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CS = 0.16


@pytest.fixture(scope="module")
def wm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03343_gb300 import build, wmibm
    build.build()
    wmibm.load()
    return wmibm


def _gpu_sgs(wm, case, dtype, vel_dtype=None):
    h = wm.Handle.from_case(case, dtype=dtype, vel_dtype=vel_dtype)
    wt = h.sgs_wall_terms(case.phi_uv, case.phi_w, case.z0)
    vd = vel_dtype or dtype
    u, v, w = (to_dev(x, vd) for x in (case.u, case.v, case.w))
    tau = [to_dev(case.tau[k], dtype) for k in inputs.TAU_NAMES]
    h.sgs_stress(u, v, w, wt, tau, cs=CS)
    torch.cuda.synchronize()
    return h, (u, v, w), wt, tau


def _oracle_sgs(oracle_mod, case, dtype, vel_dtype=None):
    rv = lambda a: to_host(to_dev(a, vel_dtype or dtype))
    rd = lambda a: to_host(to_dev(a, dtype))
    tau = {k: rd(case.tau[k]) for k in inputs.TAU_NAMES}
    oracle_mod.sgs_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_b, rv(case.u), rv(case.v),
                          rv(case.w), tau, cs=CS, kappa=inputs.KAPPA)
    return tau


def _check(tau_gpu, tau_ref, dtype):
    for k, t in zip(inputs.TAU_NAMES, tau_gpu):
        err = normwise(to_host(t), tau_ref[k])[0]
        assert err <= TOL[dtype], (k, err)


# FP32 with even nx runs the two-columns-per-thread kernel, odd nx (and FP64) the one-column march
CASES = [("ridge", (32, 32, 32), "f64"), ("ridge", (32, 32, 32), "f32"), ("cubes", (96, 48, 40), "f32"),
         ("cubes", (46, 18, 21), "f64"), ("hill", (64, 32, 24), "f32"), ("hill", (64, 32, 24), "f64"),
         ("hill", (63, 20, 17), "f32"), ("ridge", (2, 6, 9), "f32")]


@pytest.mark.parametrize("name,shape,dtype", CASES)
def test_sgs_matches_oracle(wm, oracle_mod, name, shape, dtype):
    case = inputs.make(name, shape=shape, dtype=dtype)
    h, _, _, tau = _gpu_sgs(wm, case, dtype)
    _check(tau, _oracle_sgs(oracle_mod, case, dtype), dtype)
    assert h.device_status() == wm.OK


def test_sgs_unaligned_fields_take_the_one_column_march(wm, oracle_mod):
    """Fields offset by one element from an aligned allocation (nx even, FP32): the
    pair loads would be misaligned, so the one-column march runs; same result."""
    case = inputs.hill(shape=(64, 32, 24), dtype="f32")
    h = wm.Handle.from_case(case, dtype="f32")
    wt = h.sgs_wall_terms(case.phi_uv, case.phi_w, case.z0)

    def shifted(a):
        t = to_dev(a, "f32")
        buf = torch.empty(t.numel() + 1, dtype=t.dtype, device=t.device)
        view = buf[1:].view(t.shape)
        view.copy_(t)
        return view

    u, v, w = (shifted(x) for x in (case.u, case.v, case.w))
    tau = [shifted(case.tau[k]) for k in inputs.TAU_NAMES]
    h.sgs_stress(u, v, w, wt, tau, cs=CS)
    torch.cuda.synchronize()
    _check(tau, _oracle_sgs(oracle_mod, case, "f32"), "f32")


def test_sgs_bf16_velocity(wm, oracle_mod):
    case = inputs.hill(shape=(64, 32, 24), dtype="f32")
    h, _, _, tau = _gpu_sgs(wm, case, "f32", vel_dtype="bf16")
    _check(tau, _oracle_sgs(oracle_mod, case, "f32", vel_dtype="bf16"), "f32")


def test_sgs_minimal_grid(wm, oracle_mod):
    """nz = 3 (one interior w-level), 1-wide x: the periodic neighbours are the node itself."""
    case = inputs.flat((1, 4, 3), wall_height=-1.0, lengths=(1.0, 1.0, 1.0))
    h, _, _, tau = _gpu_sgs(wm, case, "f64")
    _check(tau, _oracle_sgs(oracle_mod, case, "f64"), "f64")


def test_sgs_full_size_cubes(wm, oracle_mod):
    case = inputs.cubes(dtype="f32")
    h, _, _, tau = _gpu_sgs(wm, case, "f32")
    _check(tau, _oracle_sgs(oracle_mod, case, "f32"), "f32")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_sgs_then_wall_stress_then_force(wm, oracle_mod, dtype):
    """The stage from the velocity: SGS stress at fluid nodes, wall model at the band
    (and solid zeros), then f = -div tau, against the oracle's same chain."""
    case = inputs.ridge(shape=(48, 24, 20), dtype=dtype)
    h, (u, v, w), wt, tau = _gpu_sgs(wm, case, dtype)
    f = [torch.zeros(h.shape, dtype=h.torch_dtype, device="cuda") for _ in range(3)]
    h.wall_stress_force(u, v, w, tau, f)
    torch.cuda.synchronize()
    tau_o = _oracle_sgs(oracle_mod, case, dtype)
    rd = lambda a: to_host(to_dev(a, dtype))
    oracle_mod.wall_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b,
                           rd(case.u), rd(case.v), rd(case.w), tau_o)
    f_o = oracle_mod.force(case.grid, tau_o)
    _check(tau, tau_o, dtype)
    for c in range(3):
        assert normwise(to_host(f[c]), f_o[c])[0] <= TOL[dtype], c


def test_sgs_graph_replay(wm):
    case = inputs.cubes(shape=(64, 32, 32), dtype="f32")
    h, (u, v, w), wt, tau = _gpu_sgs(wm, case, "f32")
    ref = [to_host(t) for t in tau]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h.sgs_stress(u, v, w, wt, tau, cs=CS)
    for _ in range(4):
        for t, k in zip(tau, inputs.TAU_NAMES):
            t.copy_(to_dev(case.tau[k], "f32"))
        g.replay()
        torch.cuda.synchronize()
        for t, r in zip(tau, ref):
            assert np.array_equal(to_host(t), r)


def test_sgs_rejects_bad_coefficient(wm):
    case = inputs.ridge(shape=(16, 8, 6), dtype="f32")
    h, (u, v, w), wt, tau = _gpu_sgs(wm, case, "f32")
    with pytest.raises(wm.WmibmError, match="coefficient"):
        h.sgs_stress(u, v, w, wt, tau, cs=0.0)


def test_wall_term_markers(wm, oracle_mod):
    """Fluid nodes carry the positive wall term, band nodes -1, solid nodes -2, on the oracle's classes."""
    case = inputs.hill(shape=(64, 32, 24), dtype="f64")
    h = wm.Handle.from_case(case, dtype="f64")
    wt_uv, wt_w = (to_host(t) for t in h.sgs_wall_terms(case.phi_uv, case.phi_w, case.z0))
    cu, cw = oracle_mod.classify(case.grid, case.phi_uv, case.phi_w, case.phi_b)
    for wt, cls in ((wt_uv, cu), (wt_w, cw)):
        assert np.all(wt[cls == 1] == -1.0) and np.all(wt[cls == 2] == -2.0) and np.all(wt[cls == 0] > 0)


def _fused_vs_chain(wm, oracle_mod, case, dtype, vel_dtype=None):
    h = wm.Handle.from_case(case, dtype=dtype, vel_dtype=vel_dtype)
    wt = h.sgs_wall_terms(case.phi_uv, case.phi_w, case.z0)
    vd = vel_dtype or dtype
    u, v, w = (to_dev(x, vd) for x in (case.u, case.v, case.w))
    tau = [to_dev(case.tau[k], dtype) for k in inputs.TAU_NAMES]
    f = [torch.full(h.shape, float("nan"), dtype=h.torch_dtype, device="cuda") for _ in range(3)]
    h.wall_stress(u, v, w, tau)                     # band stresses (and solid zeros) first
    before = [t.clone() for t in tau]
    h.sgs_force(u, v, w, wt, tau, f, cs=CS)
    torch.cuda.synchronize()
    for a, b in zip(tau, before):                   # the fused call never writes the stress
        assert torch.equal(a, b)
    tau_o = _oracle_sgs(oracle_mod, case, dtype, vel_dtype)
    rv = lambda a: to_host(to_dev(a, vd))
    oracle_mod.wall_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b,
                           rv(case.u), rv(case.v), rv(case.w), tau_o)
    f_o = oracle_mod.force(case.grid, tau_o)
    for c in range(3):
        got = to_host(f[c])
        assert np.all(np.isfinite(got)), c
        assert normwise(got, f_o[c])[0] <= TOL[dtype], c
    return h, (u, v, w), wt, tau, f


FUSED = [("ridge", (32, 32, 32), "f64"), ("ridge", (40, 24, 20), "f32"), ("cubes", (96, 48, 40), "f32"),
         ("cubes", (46, 18, 21), "f64"), ("hill", (64, 32, 24), "f32"), ("hill", (70, 22, 35), "f64")]


@pytest.mark.parametrize("name,shape,dtype", FUSED)
def test_fused_stress_and_force_match_oracle(wm, oracle_mod, name, shape, dtype):
    case = inputs.make(name, shape=shape, dtype=dtype)
    h, *_ = _fused_vs_chain(wm, oracle_mod, case, dtype)
    assert h.device_status() == wm.OK


def test_fused_bf16_velocity_and_minimal_grids(wm, oracle_mod):
    _fused_vs_chain(wm, oracle_mod, inputs.hill(shape=(64, 32, 24), dtype="f32"), "f32", vel_dtype="bf16")
    # velocity noise, so that every forcing component is O(1) rather than rounding noise around 0
    _fused_vs_chain(wm, oracle_mod, inputs.flat((1, 4, 3), wall_height=-1.0, lengths=(1.0, 1.0, 1.0), sigma=0.1),
                    "f64")
    _fused_vs_chain(wm, oracle_mod, inputs.flat((5, 3, 4), wall_height=0.3, lengths=(1.0, 1.0, 1.0), sigma=0.1),
                    "f64")


def test_fused_full_size_cubes_and_chain_agreement(wm, oracle_mod):
    """The full cubes grid: fused against the oracle, and against the unfused GPU chain
    (wmibm_sgs_stress, wmibm_wall_stress, wmibm_force) within a few FP32 ulps of the
    forcing's scale."""
    case = inputs.cubes(dtype="f32")
    h, (u, v, w), wt, tau, f = _fused_vs_chain(wm, oracle_mod, case, "f32")
    tau2 = [to_dev(case.tau[k], "f32") for k in inputs.TAU_NAMES]
    f2 = [torch.zeros(h.shape, dtype=torch.float32, device="cuda") for _ in range(3)]
    h.sgs_stress(u, v, w, wt, tau2, cs=CS)
    h.wall_stress(u, v, w, tau2)
    h.force(tau2, f2)
    torch.cuda.synchronize()
    for a, b in zip(f, f2):
        assert normwise(to_host(a), to_host(b))[0] <= 1e-6


def test_fused_graph_replay(wm, oracle_mod):
    case = inputs.cubes(shape=(64, 32, 32), dtype="f32")
    h, (u, v, w), wt, tau, f = _fused_vs_chain(wm, oracle_mod, case, "f32")
    ref = [to_host(t) for t in f]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h.sgs_force(u, v, w, wt, tau, f, cs=CS)
    for _ in range(4):
        for t in f:
            t.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for t, r in zip(f, ref):
            assert np.array_equal(to_host(t), r)


def test_sgs_beside_wall_stress_on_two_streams(wm):
    """The SGS stress writes fluid entries only and the wall model band and solid
    entries only, so the two may run on two streams at once: the forcing after
    both (joined by events, also under graph capture) equals the serial chain
    bit for bit."""
    case = inputs.cubes(shape=(96, 48, 40), dtype="f32")
    h, (u, v, w), wt, tau = _gpu_sgs(wm, case, "f32")
    h.wall_stress(u, v, w, tau)
    f_ref = [torch.zeros(h.shape, dtype=torch.float32, device="cuda") for _ in range(3)]
    h.force(tau, f_ref)
    torch.cuda.synchronize()
    tau_ref = [t.clone() for t in tau]
    side = torch.cuda.Stream()
    f = [torch.zeros(h.shape, dtype=torch.float32, device="cuda") for _ in range(3)]

    def overlapped():
        cur = torch.cuda.current_stream()
        side.wait_stream(cur)
        h.sgs_stress(u, v, w, wt, tau, cs=CS)
        with torch.cuda.stream(side):
            h.wall_stress(u, v, w, tau)
        cur.wait_stream(side)
        h.force(tau, f)

    def reset():
        for t, k in zip(tau, inputs.TAU_NAMES):
            t.copy_(to_dev(case.tau[k], "f32"))
        for x in f:
            x.fill_(float("nan"))

    reset()
    overlapped()
    torch.cuda.synchronize()
    for a, b in zip(tau + f, tau_ref + f_ref):
        assert torch.equal(a, b)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        overlapped()
    for _ in range(3):
        reset()
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(tau + f, tau_ref + f_ref):
            assert torch.equal(a, b)
    assert h.device_status() == wm.OK
