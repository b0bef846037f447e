"""x-slab decomposition of one terrain over several ranks (one GPU each).

The wall-stress stage is local (Sec. 3.3: the simplified method needs only
information available to each processor), so a terrain cut into slabs along x
needs two halo exchanges per step and one small reduction:

- before the wall model, the velocity of the R = ceil((phi_c + phi_b)/dx) + 1
  x-planes beyond each edge of the slab: a band node's sample point x_c lies at
  most phi_c + phi_b from it (phi >= -phi_b on the band), and its trilinear
  stencil reaches one plane further;
- after the wall model, the six stresses of the one plane beyond each edge: the
  divergence (Eq. 18) takes central differences in x;
- the band statistics of the ranks, combined (sums and counts added, the minimum
  and maximum taken).

Each rank holds its slab padded with R planes on both sides (R >= 1: the normals
take central differences of phi across the edge).  Its handle is made with
own_x = (R, R + width): only the slab's own nodes are band, solid or body nodes,
and the halo planes carry the neighbours' values.  The padded slab is periodic
in the handle's eyes; that wrap only touches the outermost halo planes, whose
outputs are never used.

This module is host-side orchestration over the C ABI: which planes go where,
and the reduction.  The exchanges go through a communicator: TorchDistComm
(torch.distributed point-to-point: NCCL between GPUs, gloo between CPU
processes) or LocalComm (every rank in one process, copies between them).
Every exchange runs in two phases, first leftward then rightward, so that a
pair of ranks that are each other's left and right neighbours never has two
messages in flight between them.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from . import inputs

TAU_NAMES = inputs.TAU_NAMES


def halo_width(grid, phi_c, phi_b):
    """R = ceil((phi_c + phi_b) / dx) + 1 x-planes (at least one)."""
    nx, ny, nz, lx, ly, lz = grid
    dx = lx / nx
    return max(1, int(math.ceil((phi_c + phi_b) / dx - 1e-12)) + 1)


class SlabPlan:
    """Cuts the x-range [0, nx) of `grid` into `ranks` contiguous slabs (widths a
    multiple of `vec` where nx allows, so that every slab keeps the pipelined
    stencil) and pads each with `halo` planes on both sides."""

    def __init__(self, grid, ranks: int, halo: int, vec: int = 4):
        nx = int(grid[0])
        if ranks < 1:
            raise ValueError("ranks must be >= 1")
        unit = vec if nx % vec == 0 and nx // vec >= ranks else 1
        blocks = nx // unit
        if blocks < ranks:
            raise ValueError(f"nx = {nx} cannot be cut into {ranks} slabs")
        cuts = [unit * (blocks * r // ranks) for r in range(ranks + 1)]
        self.grid = tuple(grid)
        self.ranks = ranks
        self.halo = int(halo)
        self.owned = [(cuts[r], cuts[r + 1]) for r in range(ranks)]
        if min(b - a for a, b in self.owned) < self.halo:
            raise ValueError("every slab must be at least as wide as the halo")

    def width(self, r):
        a, b = self.owned[r]
        return b - a

    def local_nx(self, r):
        return self.width(r) + 2 * self.halo

    def local_grid(self, r):
        nx, ny, nz, lx, ly, lz = self.grid
        return (self.local_nx(r), ny, nz, lx / nx * self.local_nx(r), ly, lz)

    def columns(self, r):
        """Global x-index of every local x-index of slab r (periodic)."""
        a, _ = self.owned[r]
        nx = int(self.grid[0])
        return (np.arange(self.local_nx(r)) + a - self.halo) % nx

    def own_x(self, r):
        """Owned range of slab r in its local x-indices."""
        return (self.halo, self.halo + self.width(r))

    def local(self, r, a):
        """The padded slab r of a global field [k][j][i] (a copy, contiguous)."""
        return np.ascontiguousarray(np.asarray(a)[..., self.columns(r)])

    def place(self, r, local_a, global_a):
        """Writes the owned part of slab r's local field into the global field."""
        a, b = self.owned[r]
        lo, hi = self.own_x(r)
        global_a[..., a:b] = local_a[..., lo:hi]

    def left(self, r):
        return (r - 1) % self.ranks

    def right(self, r):
        return (r + 1) % self.ranks


def _edges(plan, r, width):
    """Local x-slices: (my first owned planes, my last owned planes, my left halo,
    my right halo), each `width` planes wide, next to the owned range."""
    lo, hi = plan.own_x(r)
    return (slice(lo, lo + width), slice(hi - width, hi), slice(lo - width, lo), slice(hi, hi + width))


class LocalComm:
    """Every rank in this process: an exchange copies planes between the ranks'
    arrays directly (numpy arrays or torch tensors)."""

    def __init__(self, plan: SlabPlan):
        self.plan = plan

    def exchange(self, fields_per_rank: Sequence[Sequence], width: int):
        """fields_per_rank[r] = the list of rank r's padded fields, the same fields in
        the same order on every rank.  Fills `width` halo planes on both sides."""
        plan = self.plan
        sends = []
        for r in range(plan.ranks):
            first, last, _, _ = _edges(plan, r, width)
            sends.append([(f[..., first].clone() if hasattr(f, "clone") else f[..., first].copy(),
                           f[..., last].clone() if hasattr(f, "clone") else f[..., last].copy())
                          for f in fields_per_rank[r]])
        for r in range(plan.ranks):
            _, _, lhalo, rhalo = _edges(plan, r, width)
            for q, f in enumerate(fields_per_rank[r]):
                # left halo <- the last owned planes of the left neighbour; right halo <- the
                # first owned planes of the right neighbour
                f[..., lhalo] = sends[plan.left(r)][q][1]
                f[..., rhalo] = sends[plan.right(r)][q][0]

    def reduce_stats(self, stats_per_rank):
        return combine_stats(stats_per_rank)


class TorchDistComm:
    """One rank per process over torch.distributed: point-to-point sends and
    receives of the edge planes (contiguous copies), leftward then rightward."""

    def __init__(self, plan: SlabPlan, rank: int):
        self.plan = plan
        self.rank = rank

    def _phase(self, fields, width, leftward):
        import torch
        import torch.distributed as dist
        plan, r = self.plan, self.rank
        first, last, lhalo, rhalo = _edges(plan, r, width)
        dst = plan.left(r) if leftward else plan.right(r)
        src = plan.right(r) if leftward else plan.left(r)
        bufs = []
        ops = []
        for f in fields:
            out = f[..., first if leftward else last].contiguous()
            inc = torch.empty_like(out)
            bufs.append(inc)
            ops.append(dist.P2POp(dist.isend, out, dst))
            ops.append(dist.P2POp(dist.irecv, inc, src))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for f, inc in zip(fields, bufs):
            # leftward: what arrives comes from the right neighbour's first planes -> my right halo
            f[..., rhalo if leftward else lhalo] = inc

    def exchange(self, fields: Sequence, width: int):
        if self.plan.ranks == 1:
            # a single slab is its own neighbour on both sides
            LocalComm(self.plan).exchange([list(fields)], width)
            return
        self._phase(fields, width, leftward=True)
        self._phase(fields, width, leftward=False)

    def reduce_stats(self, stats):
        """stats: this rank's [2] band records (count, sum tw, sum tw^2, min tw,
        max |U_r|, n_zclamped) as a float64 array [2, 6]; returns the combined one."""
        import torch
        import torch.distributed as dist
        s = np.asarray(stats, np.float64).reshape(2, 6)
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"      # NCCL reduces device tensors only
        add = torch.tensor(s[:, [0, 1, 2, 5]].copy(), device=dev)
        mn = torch.tensor(s[:, 3].copy(), device=dev)
        mx = torch.tensor(s[:, 4].copy(), device=dev)
        dist.all_reduce(add, op=dist.ReduceOp.SUM)
        dist.all_reduce(mn, op=dist.ReduceOp.MIN)
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        out = np.zeros((2, 6))
        out[:, [0, 1, 2, 5]] = add.cpu().numpy()
        out[:, 3] = mn.cpu().numpy()
        out[:, 4] = mx.cpu().numpy()
        return out


def combine_stats(stats_per_rank):
    """Band statistics of several slabs as one: counts, sums and clamp counts
    added, the most negative tau_w and the largest |U_r| taken.  Each entry is an
    array [2, 6] (w-band, uv-band) x (count, sum tw, sum tw^2, min tw, max |U_r|,
    n_zclamped)."""
    s = np.stack([np.asarray(x, np.float64).reshape(2, 6) for x in stats_per_rank])
    out = np.zeros((2, 6))
    for col in (0, 1, 2, 5):
        out[:, col] = s[:, :, col].sum(axis=0)
    out[:, 3] = s[:, :, 3].min(axis=0)
    out[:, 4] = s[:, :, 4].max(axis=0)
    return out


def stats_array(parsed):
    """A wmibm_band_stats pair (as Handle.parse_stats returns it) as an array [2, 6]."""
    return np.array([[p["count"], p["sum_tw"], p["sum_tw2"], p["min_tw"], p["max_ur"], p["n_zclamped"]]
                     for p in parsed], np.float64)


class SlabRank:
    """The GPU state of one slab: a handle on the padded slab that owns the slab's
    own nodes, and its fields (torch tensors on the current device)."""

    def __init__(self, plan: SlabPlan, r: int, case, dtype="f32"):
        import torch
        from . import wmibm
        self.plan, self.r = plan, r
        grid = plan.local_grid(r)
        z0 = case.z0 if np.isscalar(case.z0) else plan.local(r, case.z0)
        self.h = wmibm.Handle(grid, plan.local(r, case.phi_uv), plan.local(r, case.phi_w), z0, case.phi_c,
                              case.phi_b, dtype=dtype, own_x=plan.own_x(r))
        tdt = torch.float64 if dtype == "f64" else torch.float32
        dev = torch.device("cuda", torch.cuda.current_device())
        shape = (int(grid[2]), int(grid[1]), int(grid[0]))
        self.u, self.v, self.w = (torch.empty(shape, dtype=tdt, device=dev) for _ in range(3))
        self.tau = [torch.empty(shape, dtype=tdt, device=dev) for _ in TAU_NAMES]
        self.f = [torch.empty(shape, dtype=tdt, device=dev) for _ in range(3)]
        self.stats = self.h.new_stats()

    def load_owned(self, u, v, w, tau):
        """Owned planes from global host fields (the halo planes get NaN: the
        exchanges must fill them)."""
        import torch
        lo, hi = self.plan.own_x(self.r)
        cols = self.plan.columns(self.r)[lo:hi]
        for d, a in zip([self.u, self.v, self.w] + self.tau, [u, v, w] + [tau[k] for k in TAU_NAMES]):
            d.fill_(float("nan"))
            d[..., lo:hi] = torch.from_numpy(np.ascontiguousarray(a[..., cols])).to(d.dtype)

    def velocity(self):
        return [self.u, self.v, self.w]


def step(ranks: List[SlabRank], comm):
    """One wall stress + force step of every slab with LocalComm (all slabs in this
    process): velocity halo, wall model, stress halo, forcing; returns the
    combined band statistics [2, 6]."""
    plan = ranks[0].plan
    comm.exchange([rk.velocity() for rk in ranks], plan.halo)
    for rk in ranks:
        rk.h.wall_stress(rk.u, rk.v, rk.w, rk.tau, rk.stats)
    comm.exchange([rk.tau for rk in ranks], 1)
    for rk in ranks:
        rk.h.force(rk.tau, rk.f)
    return comm.reduce_stats([stats_array(rk.h.parse_stats(rk.stats)) for rk in ranks])


def step_rank(rk: SlabRank, comm: TorchDistComm):
    """The same step for one rank of a torch.distributed job."""
    comm.exchange(rk.velocity(), rk.plan.halo)
    rk.h.wall_stress(rk.u, rk.v, rk.w, rk.tau, rk.stats)
    comm.exchange(rk.tau, 1)
    rk.h.force(rk.tau, rk.f)
    return comm.reduce_stats(stats_array(rk.h.parse_stats(rk.stats)))
