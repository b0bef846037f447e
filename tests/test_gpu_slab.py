"""The x-slab decomposition on the GPU: each slab a handle that owns its own
x-range of a padded slab (wmibm_opts.own_x0/own_x1), the slabs stepped one
after another in this process with their halos copied between them (no kernel
waits on another).  The owned results, put together, match the whole-domain
oracle and the whole-domain GPU handle; every slab's band set is the whole
domain's restricted to it; the combined band statistics are the whole domain's
(Sec. 3.3: the simplified method needs only information available to each
processor)."""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import TOL, assert_stats_close, normwise, oracle_lists, oracle_step, to_host

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
    "cubes": lambda: inputs.cubes(shape=(96, 48, 40)),
    "hill": lambda: inputs.hill(shape=(128, 48, 40)),
    "ensemble": lambda: inputs.ensemble_member(11, shape=(128, 64, 32)),
}


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("ranks", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_slabs_match_the_whole_domain(wm, oracle_mod, name, ranks, dtype):
    from paper_2006_03343_gb300 import slab
    case = CASES[name]()
    R = slab.halo_width(case.grid, case.phi_c, case.phi_b)
    plan = slab.SlabPlan(case.grid, ranks, R)
    rks = [slab.SlabRank(plan, r, case, dtype) for r in range(ranks)]
    for rk in rks:
        rk.load_owned(case.u, case.v, case.w, case.tau)
    stats = slab.step(rks, slab.LocalComm(plan))
    torch.cuda.synchronize()
    tau = {k: np.full(case.shape, np.nan) for k in inputs.TAU_NAMES}
    f = [np.full(case.shape, np.nan) for _ in range(3)]
    for r, rk in enumerate(rks):
        for k, t in zip(inputs.TAU_NAMES, rk.tau):
            plan.place(r, to_host(t), tau[k])
        for c in range(3):
            plan.place(r, to_host(rk.f[c]), f[c])
        assert rk.h.device_status() == wm.OK
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    for k in inputs.TAU_NAMES:
        assert normwise(tau[k], tau_o[k])[0] <= TOL[dtype], (k, name, ranks)
    for c in range(3):
        assert normwise(f[c], f_o[c])[0] <= TOL[dtype], (c, name, ranks)
    parsed = np.zeros(2, dtype=wm.STATS_DTYPE)
    for b in range(2):
        parsed[b] = (int(stats[b, 0]), stats[b, 1], stats[b, 2], stats[b, 3], stats[b, 4], int(stats[b, 5]))
    assert_stats_close(parsed, st_o, dtype)
    # band, solid and body sets: the slabs' own nodes, in global numbering, are the whole domain's
    ref = oracle_lists(oracle_mod, case)
    nx, ny, _ = case.grid[:3]
    for which in range(6):
        got = []
        for r, rk in enumerate(rks):
            loc = rk.h.export_list(which).astype(np.int64)
            lnx = plan.local_nx(r)
            k, rem = np.divmod(loc, lnx * ny)
            j, i = np.divmod(rem, lnx)
            got.append((k * ny + j) * nx + plan.columns(r)[i])
        assert np.array_equal(np.sort(np.concatenate(got)), ref[which]), (name, which)
    # and the whole-domain GPU handle
    h = wm.Handle.from_case(case, dtype=dtype)
    from parity_util import gpu_step
    tau_g, f_g, _, _ = gpu_step(h, case, dtype)
    for c in range(3):
        assert normwise(f[c], f_g[c])[0] <= TOL[dtype]
    h.close()


def test_slab_halo_and_owned_range_validation(wm):
    from paper_2006_03343_gb300 import slab
    case = inputs.hill(shape=(64, 32, 24))
    with pytest.raises(wm.WmibmError):
        wm.Handle(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b, own_x=(10, 70))
    with pytest.raises(wm.WmibmError):
        wm.Handle(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b, own_x=(20, 20))
    h = wm.Handle(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b, own_x=(16, 48))
    band = h.export_list(wm.LIST_BAND_W) % 64
    assert band.size and band.min() >= 16 and band.max() < 48
    h.close()
