"""GPU adjoint (wmibm_set_log_z0, wmibm_backward and the autograd wrapper) against
the FP64 oracle's adjoint, against central differences of the GPU forward, and
for determinism.  L = sum(g . f) over the three forcing components."""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import TOL, normwise, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL = (40, 24, 22)     # several tiles with ragged edges; the oracle finishes in well under a second


@pytest.fixture(scope="module")
def wm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03343_gb300 import build, wmibm
    build.build()
    wmibm.load()
    return wmibm


def _setup(wm, shape, dtype, vel_dtype=None):
    case, g = inputs.adjoint_case(shape=shape, dtype=dtype)
    s = np.log(case.z0)
    h = wm.Handle.from_case(case, dtype=dtype, vel_dtype=vel_dtype)
    dev = dict(u=to_dev(case.u, vel_dtype or dtype), v=to_dev(case.v, vel_dtype or dtype),
               w=to_dev(case.w, vel_dtype or dtype), s=to_dev(s, dtype), g=[to_dev(x, dtype) for x in g])
    h.set_log_z0(dev["s"])
    return case, g, s, h, dev


def _gpu_grad(h, dev, dtype, with_ds=True):
    shp = h.shape
    tdt = torch.float64 if dtype == "f64" else torch.float32
    out = [torch.empty(shp, dtype=tdt, device="cuda") for _ in range(4)]
    h.backward(dev["g"], (dev["u"], dev["v"], dev["w"]), out[0], out[1], out[2], out[3] if with_ds else None)
    torch.cuda.synchronize()
    return out


def _oracle_grad(oracle, case, g, s, u=None, v=None, w=None):
    u = case.u if u is None else u
    v = case.v if v is None else v
    w = case.w if w is None else w
    return oracle.adjoint(case.grid, case.phi_uv, case.phi_w, s, case.phi_c, case.phi_b, u, v, w, g)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_backward_matches_oracle_adjoint(wm, oracle_mod, dtype):
    case, g, s, h, dev = _setup(wm, SMALL, dtype)
    got = [to_host(t) for t in _gpu_grad(h, dev, dtype)]
    # the oracle sees the same (rounded) inputs the GPU saw
    rd = lambda a: to_host(to_dev(a, dtype))
    ref = _oracle_grad(oracle_mod, case, [rd(x) for x in g], rd(s), rd(case.u), rd(case.v), rd(case.w))
    for name, a, b in zip(("du", "dv", "dw", "dlogz0"), got, ref):
        assert np.abs(b).max() > 0, name
        err = normwise(a, b)[0]
        assert err <= TOL[dtype], (name, err)
        # the support is the same: nodes the oracle leaves at zero stay zero
        assert np.all(a[b == 0] == 0), name
    assert h.device_status() == wm.OK


def test_forward_with_log_z0_matches_oracle(wm, oracle_mod):
    """Forward wall stress with the per-cell ln z0 field (FP64) against the oracle's log mode."""
    case, g, s, h, dev = _setup(wm, SMALL, "f64")
    tau = [to_dev(case.tau[k], "f64") for k in inputs.TAU_NAMES]
    st = h.new_stats()
    h.wall_stress(dev["u"], dev["v"], dev["w"], tau, st)
    torch.cuda.synchronize()
    ref = {k: t.copy() for k, t in case.tau.items()}
    oracle_mod.wall_stress(case.grid, case.phi_uv, case.phi_w, None, case.phi_c, case.phi_b, case.u, case.v,
                           case.w, ref, logz0=s)
    for k, t in zip(inputs.TAU_NAMES, tau):
        assert normwise(to_host(t), ref[k])[0] <= TOL["f64"], k


def test_backward_is_deterministic(wm):
    case, g, s, h, dev = _setup(wm, SMALL, "f32")
    a = [to_host(t) for t in _gpu_grad(h, dev, "f32")]
    b = [to_host(t) for t in _gpu_grad(h, dev, "f32")]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def _gpu_loss_delta(h, dev, case, which, idx, step):
    """sum(g . (f(x + step e) - f(x - step e))) with the GPU FP64 forward (the forward is
    local, so the difference of the two fields is exact almost everywhere)."""
    fs = []
    for sign in (1, -1):
        x = {k: dev[k].clone() for k in ("u", "v", "w", "s")}
        x[which].view(-1)[idx] += sign * step
        h.set_log_z0(x["s"])
        tau = [to_dev(case.tau[k], "f64") for k in inputs.TAU_NAMES]
        f = [torch.empty(h.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
        h.wall_stress_force(x["u"], x["v"], x["w"], tau, f)
        fs.append(f)
    h.set_log_z0(dev["s"])
    return float(sum(torch.sum(gi * (a - b)) for gi, a, b in zip(dev["g"], fs[0], fs[1])).item())


@pytest.mark.parametrize("which", ["u", "v", "w", "s"])
def test_backward_matches_central_differences_full_size(wm, which):
    """256 x 128 x 128 multi-hill terrain, FP64: dL/dx at entries of the 32^3 block at
    offset (64, 32, 0) (it holds surface nodes) equals the central difference."""
    case, g, s, h, dev = _setup(wm, inputs.ADJOINT_SHAPE, "f64")
    grads = dict(zip(("u", "v", "w", "s"), _gpu_grad(h, dev, "f64")))
    grad = grads[which]
    block = grad[0:32, 32:64, 64:96]
    gb = to_host(block)
    assert np.abs(gb).max() > 0
    nz_, ny_, nx_ = h.shape
    flat = np.argsort(np.abs(gb).ravel())[::-1][:8]
    rng = np.random.default_rng(5)
    picks = list(flat) + list(rng.choice(gb.size, size=4, replace=False))
    scale = np.abs(gb).max()
    step = 1e-6
    for q in picks:
        k, j, i = np.unravel_index(int(q), gb.shape)
        idx = (k * ny_ + (j + 32)) * nx_ + (i + 64)
        fd = _gpu_loss_delta(h, dev, case, which, idx, step) / (2 * step)
        assert abs(fd - gb[k, j, i]) <= 1e-6 * scale, (which, (k, j, i), fd, gb[k, j, i])


def test_full_size_backward_matches_oracle(wm, oracle_mod):
    """The whole 256 x 128 x 128 problem in FP32 against the FP64 oracle adjoint."""
    case, g, s, h, dev = _setup(wm, inputs.ADJOINT_SHAPE, "f32")
    got = [to_host(t) for t in _gpu_grad(h, dev, "f32")]
    rd = lambda a: to_host(to_dev(a, "f32"))
    ref = _oracle_grad(oracle_mod, case, [rd(x) for x in g], rd(s), rd(case.u), rd(case.v), rd(case.w))
    for name, a, b in zip(("du", "dv", "dw", "dlogz0"), got, ref):
        assert normwise(a, b)[0] <= TOL["f32"], name


def test_autograd_matches_backward(wm):
    from paper_2006_03343_gb300 import autograd
    case, g, s, h, dev = _setup(wm, SMALL, "f64")
    u, v, w, ls = (dev[k].clone().requires_grad_(True) for k in ("u", "v", "w", "s"))
    tau = [to_dev(case.tau[k], "f64") for k in inputs.TAU_NAMES]
    tau_before = [t.clone() for t in tau]
    fx, fy, fz = autograd.wall_stress_force(h, u, v, w, ls, tau)
    loss = sum(torch.sum(gi * fi) for gi, fi in zip(dev["g"], (fx, fy, fz)))
    loss.backward()
    ref = _gpu_grad(h, dev, "f64")
    for got, r in zip((u.grad, v.grad, w.grad, ls.grad), ref):
        assert torch.equal(got, r)
    for a, b in zip(tau, tau_before):
        assert torch.equal(a, b)           # the given stresses are not modified
    # directional derivative of the autograd loss
    d = [torch.randn_like(x) for x in (u, v, w)] + [0.1 * torch.randn_like(ls)]
    hstep = 1e-6
    vals = []
    for sign in (1, -1):
        with torch.no_grad():
            out = autograd.wall_stress_force(h, u + sign * hstep * d[0], v + sign * hstep * d[1],
                                             w + sign * hstep * d[2], ls + sign * hstep * d[3], tau)
            vals.append(sum(torch.sum(gi * fi) for gi, fi in zip(dev["g"], out)))
    fd = float((vals[0] - vals[1]).item()) / (2 * hstep)
    ad = float(sum(torch.sum(a * b) for a, b in zip((u.grad, v.grad, w.grad, ls.grad), d)).item())
    assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), (fd, ad)


def test_backward_bf16_velocity(wm, oracle_mod):
    """BF16 velocity storage: gradients in FP32 against the oracle on the BF16-rounded velocity."""
    case, g, s, h, dev = _setup(wm, SMALL, "f32", vel_dtype="bf16")
    got = [to_host(t) for t in _gpu_grad(h, dev, "f32")]
    rv = lambda a: to_host(to_dev(a, "bf16"))
    rd = lambda a: to_host(to_dev(a, "f32"))
    ref = _oracle_grad(oracle_mod, case, [rd(x) for x in g], rd(s), rv(case.u), rv(case.v), rv(case.w))
    for name, a, b in zip(("du", "dv", "dw", "dlogz0"), got, ref):
        assert normwise(a, b)[0] <= TOL["f32"], name


def test_backward_without_log_field_and_no_band(wm):
    """No ln z0 field: the derivative is taken at the init roughness; an all-fluid grid
    (no band) gives zero gradients."""
    case, g, s, h, dev = _setup(wm, SMALL, "f64")
    h.set_log_z0(None)
    a = _gpu_grad(h, dev, "f64")
    h.set_log_z0(dev["s"])
    b = _gpu_grad(h, dev, "f64")
    for x, y in zip(a, b):
        assert normwise(to_host(x), to_host(y))[0] <= 1e-12
    flat = inputs.flat((16, 8, 10), wall_height=-1.0, dtype="f64")
    hf = wm.Handle.from_case(flat, dtype="f64")
    assert hf.list_size(wm.LIST_BAND_W) == 0 and hf.list_size(wm.LIST_BAND_UV) == 0
    z = lambda: torch.zeros(hf.shape, dtype=torch.float64, device="cuda")
    gs = [torch.ones(hf.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    outs = [z() + 7 for _ in range(4)]
    hf.backward(gs, (z(), z(), z()), *outs)
    torch.cuda.synchronize()
    for o in outs:
        assert float(o.abs().max()) == 0.0
