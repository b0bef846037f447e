"""Pins of the oracle's hand-derived adjoint (L = sum g . f over the three forcing
components, per-cell roughness s = ln z0): the transpose identity of the
divergence, central finite differences of L through the oracle's forward at
sampled entries, and a whole-field directional derivative.  None of these
compares the adjoint with itself: the forward pass (wall stress of Sec. 3.3,
f = -div tau of Eqs. 15-16 and Eq. 18) is the reference."""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

H = 1e-6          # central-difference step (FP64)
SHAPE = (32, 24, 20)


@pytest.fixture(scope="module")
def problem():
    case, g = inputs.adjoint_case(shape=SHAPE, dtype="f64")
    return case, g, np.ascontiguousarray(np.log(case.z0))


def loss(oracle, case, g, u, v, w, logz0):
    tau = {k: t.copy() for k, t in case.tau.items()}
    oracle.wall_stress(case.grid, case.phi_uv, case.phi_w, None, case.phi_c, case.phi_b, u, v, w, tau,
                       logz0=logz0)
    f = oracle.force(case.grid, tau)
    return float(sum(np.sum(gi * fi) for gi, fi in zip(g, f)))


def test_force_adjoint_is_the_transpose(oracle_mod):
    """<g, D tau> = <D^T g, tau> for random tau and g (exact up to rounding)."""
    rng = np.random.default_rng(11)
    grid = (10, 7, 6, 2.0, 1.5, 1.0)
    shp = (6, 7, 10)
    tau = {k: rng.standard_normal(shp) for k in inputs.TAU_NAMES}
    g = [rng.standard_normal(shp) for _ in range(3)]
    f = oracle_mod.force(grid, tau)
    gam = oracle_mod.force_adjoint(grid, g)
    lhs = sum(float(np.sum(a * b)) for a, b in zip(g, f))
    rhs = sum(float(np.sum(gam[k] * tau[k])) for k in inputs.TAU_NAMES)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    # one stress entry at a time: column p of D^T is the response of f to a unit tau at p
    for name in ("txx", "tzz", "txz", "tyz"):
        unit = {k: np.zeros(shp) for k in inputs.TAU_NAMES}
        unit[name][3, 2, 9] = 1.0
        fu = oracle_mod.force(grid, unit)
        assert np.isclose(sum(float(np.sum(a * b)) for a, b in zip(g, fu)), gam[name][3, 2, 9], rtol=0, atol=1e-12)


def test_log_mode_forward_matches_z0_field(oracle_mod, problem):
    """The forward with ln z0 per cell equals the one with z0 per cell up to the rounding of the log."""
    case, _, s = problem
    ta = {k: t.copy() for k, t in case.tau.items()}
    tb = {k: t.copy() for k, t in case.tau.items()}
    oracle_mod.wall_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b,
                           case.u, case.v, case.w, ta)
    oracle_mod.wall_stress(case.grid, case.phi_uv, case.phi_w, None, case.phi_c, case.phi_b,
                           case.u, case.v, case.w, tb, logz0=s)
    for k in inputs.TAU_NAMES:
        scale = max(np.abs(ta[k]).max(), 1e-30)
        assert np.abs(ta[k] - tb[k]).max() <= 1e-13 * scale, k


def _samples(grad, rng, n_top=10, n_rand=6, n_zero=3):
    flat = np.abs(grad).ravel()
    order = np.argsort(flat)[::-1]
    top = list(order[:n_top])
    nz = np.nonzero(flat)[0]
    rand = list(rng.choice(nz, size=min(n_rand, nz.size), replace=False)) if nz.size else []
    zero = np.nonzero(flat == 0)[0]
    zer = list(rng.choice(zero, size=min(n_zero, zero.size), replace=False)) if zero.size else []
    return sorted(set(int(i) for i in top + rand + zer))


@pytest.mark.parametrize("which", ["u", "v", "w", "logz0"])
def test_adjoint_matches_central_differences(oracle_mod, problem, which):
    """dL/dx at sampled entries (largest, random nonzero, and zero ones) equals the
    central difference [L(x + h e) - L(x - h e)] / 2h of the forward."""
    case, g, s = problem
    du, dv, dw, ds = oracle_mod.adjoint(case.grid, case.phi_uv, case.phi_w, s, case.phi_c, case.phi_b,
                                        case.u, case.v, case.w, g)
    grad = {"u": du, "v": dv, "w": dw, "logz0": ds}[which]
    assert np.abs(grad).max() > 0
    rng = np.random.default_rng(7)
    scale = np.abs(grad).max()
    fields = {"u": case.u, "v": case.v, "w": case.w, "logz0": s}
    for idx in _samples(grad, rng):
        vals = {}
        for sign in (1, -1):
            x = {k: a.copy() for k, a in fields.items()}
            x[which].ravel()[idx] += sign * H
            vals[sign] = loss(oracle_mod, case, g, x["u"], x["v"], x["w"], x["logz0"])
        fd = (vals[1] - vals[-1]) / (2 * H)
        assert abs(fd - grad.ravel()[idx]) <= 2e-6 * scale, (which, idx, fd, grad.ravel()[idx])


def test_directional_derivative(oracle_mod, problem):
    """<grad L, d> = [L(x + h d) - L(x - h d)] / 2h for one random direction in (u, v, w, ln z0)."""
    case, g, s = problem
    du, dv, dw, ds = oracle_mod.adjoint(case.grid, case.phi_uv, case.phi_w, s, case.phi_c, case.phi_b,
                                        case.u, case.v, case.w, g)
    rng = np.random.default_rng(9)
    d = [rng.standard_normal(case.u.shape) for _ in range(3)] + [0.1 * rng.standard_normal(s.shape)]
    ad = sum(float(np.sum(a * b)) for a, b in zip((du, dv, dw, ds), d))
    lp = loss(oracle_mod, case, g, case.u + H * d[0], case.v + H * d[1], case.w + H * d[2], s + H * d[3])
    lm = loss(oracle_mod, case, g, case.u - H * d[0], case.v - H * d[1], case.w - H * d[2], s - H * d[3])
    fd = (lp - lm) / (2 * H)
    assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), (fd, ad)


def test_adjoint_zero_away_from_the_band(oracle_mod, problem):
    """Only velocity nodes inside some interpolation stencil and only band cells get gradient."""
    case, g, s = problem
    du, dv, dw, ds = oracle_mod.adjoint(case.grid, case.phi_uv, case.phi_w, s, case.phi_c, case.phi_b,
                                        case.u, case.v, case.w, g)
    cu, cw = oracle_mod.classify(case.grid, case.phi_uv, case.phi_w, case.phi_b)
    band_cell = (cu == 1) | (cw == 1)
    assert np.all(ds[~band_cell] == 0)
    # the sample point lies at most phi_c + phi_b above the node along n, so nothing
    # above the band's highest level plus that reach (and one stencil level) is touched
    dz = case.grid[5] / (case.grid[2] - 1)
    kmax = int(np.nonzero(band_cell.any(axis=(1, 2)))[0].max())
    reach = int(np.ceil((case.phi_c + case.phi_b) / dz)) + 2
    for a in (du, dv, dw):
        assert np.all(a[kmax + reach:] == 0)
