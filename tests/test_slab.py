"""The x-slab decomposition's host logic on CPU ranks (gloo, world size 2), with
the FP64 oracle standing in for each rank's kernels: slabs padded with the halo
of ceil((phi_c + phi_b)/dx) + 1 planes, the velocity halo exchanged before the
wall model and one stress plane after it, owned results gathered and compared
with the whole-domain oracle; the band sets of the slabs are those of the whole
domain; the statistics reduction.  (The paper's statement that the simplified
method needs only information available to each processor: Sec. 3.3.)"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    sys.path.insert(0, ROOT)
    from paper_2006_03343_gb300 import inputs
    if name == "hill":
        return inputs.hill(shape=(48, 24, 20), seed=9, dtype="f64")
    return inputs.ensemble_member(7, shape=(64, 16, 24), dtype="f64")


def _rank(rank, world, port, name, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2006_03343_gb300 import inputs, slab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = _case(name)
        R = slab.halo_width(case.grid, case.phi_c, case.phi_b)
        plan = slab.SlabPlan(case.grid, world, R)
        comm = slab.TorchDistComm(plan, rank)
        grid = plan.local_grid(rank)
        lo, hi = plan.own_x(rank)
        cols = plan.columns(rank)

        def padded(a):
            x = np.full(a.shape[:2] + (plan.local_nx(rank),), np.nan)
            x[..., lo:hi] = a[..., cols[lo:hi]]
            return x

        u, v, w = (torch.from_numpy(padded(a)) for a in (case.u, case.v, case.w))
        tau = [torch.from_numpy(padded(case.tau[k])) for k in inputs.TAU_NAMES]
        comm.exchange([u, v, w], R)                  # velocity halo
        assert not any(torch.isnan(t).any() for t in (u, v, w))
        phi_uv, phi_w = plan.local(rank, case.phi_uv), plan.local(rank, case.phi_w)
        td = {k: t.numpy() for k, t in zip(inputs.TAU_NAMES, tau)}
        z0 = case.z0 if np.isscalar(case.z0) else plan.local(rank, case.z0)
        oracle.wall_stress(grid, phi_uv, phi_w, z0, case.phi_c, case.phi_b, u.numpy(), v.numpy(), w.numpy(), td)
        comm.exchange(tau, 1)                        # one stress plane
        f = oracle.force(grid, {k: t.numpy() for k, t in zip(inputs.TAU_NAMES, tau)})
        cu, cw = oracle.classify(grid, phi_uv, phi_w, case.phi_b)
        out[rank] = dict(tau=[t.numpy()[..., lo:hi].copy() for t in tau], f=[a[..., lo:hi].copy() for a in f],
                         cls_uv=cu[..., lo:hi].copy(), cls_w=cw[..., lo:hi].copy(), owned=plan.owned[rank])
        # the statistics reduction across the two ranks
        mine = np.array([[10 + rank, -1.0 - rank, 2.0, -0.5 * (rank + 1), 3.0 - rank, rank],
                         [5, -2.0, 4.0 + rank, -0.25, 1.5 + rank, 2 * rank]])
        out[f"stats{rank}"] = comm.reduce_stats(mine)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["hill", "ensemble"])
def test_two_gloo_ranks_match_the_whole_domain(oracle_mod, name):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_2006_03343_gb300 import inputs, slab
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, name, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    case = _case(name)
    tau_o = {k: case.tau[k].copy() for k in inputs.TAU_NAMES}
    oracle_mod.wall_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b, case.u, case.v,
                           case.w, tau_o)
    f_o = oracle_mod.force(case.grid, tau_o)
    cu, cw = oracle_mod.classify(case.grid, case.phi_uv, case.phi_w, case.phi_b)
    for r in range(2):
        a, b = out[r]["owned"]
        for q, k in enumerate(inputs.TAU_NAMES):
            ref = tau_o[k][..., a:b]
            err = np.max(np.abs(out[r]["tau"][q] - ref)) / max(np.max(np.abs(tau_o[k])), 1e-300)
            assert err <= 1e-12, (r, k, err)
        for c in range(3):
            ref = f_o[c][..., a:b]
            err = np.max(np.abs(out[r]["f"][c] - ref)) / max(np.max(np.abs(f_o[c])), 1e-300)
            assert err <= 1e-12, (r, c, err)
        assert np.array_equal(out[r]["cls_uv"], cu[..., a:b]) and np.array_equal(out[r]["cls_w"], cw[..., a:b])
    s0, s1 = out["stats0"], out["stats1"]
    assert np.array_equal(s0, s1)
    assert np.array_equal(s0[:, 0], [21, 10]) and np.array_equal(s0[:, 5], [1, 2])
    assert s0[0, 1] == -3.0 and s0[1, 2] == 9.0
    assert s0[0, 3] == -1.0 and s0[1, 3] == -0.25 and s0[0, 4] == 3.0 and s0[1, 4] == 2.5


def test_plan_cuts_and_halo():
    sys.path.insert(0, ROOT)
    from paper_2006_03343_gb300 import slab
    grid = (64, 8, 10, 6.4, 1.0, 1.0)               # dx = 0.1, dz = 1/9
    assert slab.halo_width(grid, 0.15, 0.05) == 3    # ceil(0.2 / 0.1) + 1
    plan = slab.SlabPlan(grid, 3, 3)
    assert [b - a for a, b in plan.owned] == [20, 20, 24] and all(a % 4 == 0 for a, _ in plan.owned)
    assert plan.owned[0][0] == 0 and plan.owned[-1][1] == 64
    assert list(plan.columns(0)[:4]) == [61, 62, 63, 0]
    assert plan.own_x(1) == (3, 23) and plan.local_nx(1) == 26
    with pytest.raises(ValueError):
        slab.SlabPlan(grid, 40, 3)
    s = slab.combine_stats([np.array([[1, -1.0, 1.0, -1.0, 2.0, 0], [0, 0, 0, 0, 0, 0]]),
                            np.array([[2, -3.0, 5.0, -2.5, 1.0, 1], [1, -1.0, 1.0, -1.0, 1.0, 1]])])
    assert s[0].tolist() == [3, -4.0, 6.0, -2.5, 2.0, 1] and s[1].tolist() == [1, -1.0, 1.0, -1.0, 1.0, 1]


def test_local_comm_fills_every_halo_plane():
    sys.path.insert(0, ROOT)
    from paper_2006_03343_gb300 import slab
    grid = (32, 2, 3, 3.2, 1.0, 1.0)
    plan = slab.SlabPlan(grid, 3, 2)
    glob = np.arange(3 * 2 * 32, dtype=np.float64).reshape(3, 2, 32)
    fields = []
    for r in range(3):
        x = plan.local(r, glob)
        lo, hi = plan.own_x(r)
        x[..., :lo] = np.nan
        x[..., hi:] = np.nan
        fields.append([x])
    slab.LocalComm(plan).exchange(fields, 2)
    for r in range(3):
        assert np.array_equal(fields[r][0], plan.local(r, glob))
