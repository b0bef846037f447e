"""Shared helpers of the GPU parity tests: run a case through the C ABI and
through the FP64 oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np

from paper_2006_03343_gb300 import inputs

TOL = {"f64": 1e-12, "f32": 1e-5}
STATS_TOL = {"f64": 1e-11, "f32": 1e-5}


def normwise(gpu, ref):
    """max |gpu - ref| / max |ref| (0/0 counts as 0) and the RMS of the error; a
    non-finite GPU entry makes the error infinite."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if gpu.size and not np.all(np.isfinite(gpu)):
        return float("inf"), float("inf")
    den = np.max(np.abs(ref)) if ref.size else 0.0
    err = np.max(np.abs(gpu - ref)) if ref.size else 0.0
    rms = float(np.sqrt(np.mean((gpu - ref) ** 2))) if ref.size else 0.0
    if den == 0.0:
        return float(err), rms
    return float(err / den), rms


def torch_dtype(name):
    import torch
    return {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[name]


def to_dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch_dtype(dtype)).contiguous()


def to_host(t):
    import torch
    return t.detach().to(torch.float64).cpu().numpy()


def rounded(a, dtype):
    """The float64 values the GPU actually sees after storage in `dtype`."""
    import torch
    if dtype == "f64":
        return np.ascontiguousarray(a)
    return to_host(torch.from_numpy(np.ascontiguousarray(a)).to(torch_dtype(dtype)))


def oracle_step(oracle, case, u=None, v=None, w=None, tau=None):
    """Oracle wall stress + force on (possibly pre-rounded) inputs."""
    u = case.u if u is None else u
    v = case.v if v is None else v
    w = case.w if w is None else w
    tau = {k: (case.tau[k] if tau is None else tau[k]).copy() for k in inputs.TAU_NAMES}
    stats = oracle.wall_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b, u, v, w, tau)
    f = oracle.force(case.grid, tau)
    return tau, f, stats


def poisoned_tau(case):
    """The case's stresses with NaN at every band and solid node (the entries the
    wall model writes), so that an entry the GPU leaves unwritten shows up."""
    out = {}
    for k in inputs.TAU_NAMES:
        a = case.tau[k].copy()
        if inputs.TAU_ON_W[k]:
            a[case.phi_w <= case.phi_b] = np.nan
        else:
            a[case.phi_uv <= 2.0 * case.phi_b] = np.nan
        out[k] = a
    return out


def gpu_step(handle, case, dtype, vel_dtype=None, offset=0):
    """wall_stress then force through the C ABI; `offset` shifts every device
    buffer by that many elements (misaligned pointers take the scalar path).  The
    forcing starts as NaN everywhere and the stress as NaN where the wall model
    writes it."""
    import torch
    vel_dtype = vel_dtype or dtype

    def dev(a, dt):
        if offset == 0:
            return to_dev(a, dt)
        flat = torch.empty(a.size + offset, dtype=torch_dtype(dt), device="cuda")
        view = flat[offset:].view(a.shape)
        view.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(torch_dtype(dt)))
        return view

    u, v, w = (dev(x, vel_dtype) for x in (case.u, case.v, case.w))
    pt = poisoned_tau(case)
    tau = [dev(pt[k], dtype) for k in inputs.TAU_NAMES]
    f = [dev(np.full(case.shape, np.nan), dtype) for _ in range(3)]
    stats = handle.new_stats()
    handle.wall_stress(u, v, w, tau, stats)
    handle.force(tau, f)
    torch.cuda.synchronize()
    return ({k: to_host(t) for k, t in zip(inputs.TAU_NAMES, tau)}, tuple(to_host(t) for t in f),
            handle.parse_stats(stats), (u, v, w, tau, f))


def oracle_lists(oracle, case):
    cu, cw = oracle.classify(case.grid, case.phi_uv, case.phi_w, case.phi_b)
    flat_u, flat_w = cu.ravel(), cw.ravel()
    return [np.nonzero(flat_w == 1)[0], np.nonzero(flat_u == 1)[0], np.nonzero(flat_w == 2)[0],
            np.nonzero(flat_u == 2)[0], np.nonzero(case.phi_w.ravel() <= 0)[0],
            np.nonzero(case.phi_uv.ravel() <= 0)[0]]


def assert_stats_close(gs, os_, dtype):
    tol = STATS_TOL[dtype]
    for b in range(2):
        assert gs[b]["count"] == int(os_[b, 0])
        assert gs[b]["n_zclamped"] == int(os_[b, 5])
        for col, name in ((1, "sum_tw"), (2, "sum_tw2"), (3, "min_tw"), (4, "max_ur")):
            ref = os_[b, col]
            got = gs[b][name]
            scale = max(abs(ref), 1e-30)
            assert abs(got - ref) <= tol * scale + 1e-300, (b, name, got, ref)


def gpu_fused(handle, case, dtype, vel_dtype=None, with_stats=True):
    """The fused wall stress + force pass through the C ABI (outputs poisoned with
    NaN as in gpu_step)."""
    import torch
    vel_dtype = vel_dtype or dtype
    u, v, w = (to_dev(x, vel_dtype) for x in (case.u, case.v, case.w))
    pt = poisoned_tau(case)
    tau = [to_dev(pt[k], dtype) for k in inputs.TAU_NAMES]
    f = [to_dev(np.full(case.shape, np.nan), dtype) for _ in range(3)]
    stats = handle.new_stats() if with_stats else None
    handle.wall_stress_force(u, v, w, tau, f, stats)
    torch.cuda.synchronize()
    st = handle.parse_stats(stats) if with_stats else None
    return ({k: to_host(t) for k, t in zip(inputs.TAU_NAMES, tau)}, tuple(to_host(t) for t in f), st)
