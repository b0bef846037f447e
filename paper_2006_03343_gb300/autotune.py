"""Autotuner of the stencil launch shape, for one terrain and for a batch.

One terrain: times wall stress + force (wmibm_wall_stress_force) of a handle
over its forms -- one cooperative launch with the wall phase inside the
pipelined stencil (a share in every block, dedicated wall blocks, the band
records as interleaved pipeline stages, or wall warps beside the producer and
consumers of every block), or the wall kernel followed by the stencil -- and a
grid of tile shapes (rows per strip, shared-memory stages, consumer warps,
warps and blocks per SM of the wall kernel, band records per wall stage, units
per take of the dynamic dispensing) with CUDA
events on the launching stream (L2 flushed before every timed call), keeps the
fastest, applies it to the handle and caches it in a JSON file keyed by GPU,
precision and grid size.  A single-launch form is taken only when it beats the
best two-launch form by more than 2 %; closer than that the two are a tie and
the two-launch form is kept.

A batch: the same for wmibm_batch_wall_stress_force over the batch forms (one
cooperative launch with wall warps or with interleaved wall stages, or the
batch wall kernel then the batch stencil), rows per strip of the widest
members, stages, consumer warps, wall warps and the dynamic dispensing; cached
by the members' grid sizes.

Before a shape is kept, its forcing is compared with the forcing of the
library's default shape on the same inputs: a shape whose result differs by
more than 1e-6 (FP32) or 1e-13 (FP64) of the largest value is rejected and the
next fastest is taken.  The timed calls go through the C ABI like any other
call; nothing here computes anything of the method.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
import time

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "tuning.json")

ROWS = (1, 2, 4)
STAGES = (2, 3, 4, 5, 6)
CONSUMERS = (2, 3, 4, 6, 8)
WALL_WARPS = (4, 8)
WALL_CHUNK_PER_THREAD = (0, 4)     # band records per consumer thread and wall stage (0: the library's default)
WALL_WARPS_IN_BLOCK = (1, 2, 3)     # wall warps beside the producer and consumers (force_path 6)
DYN_CHUNKS = (0, 16)                # units per take of the dynamic dispensing (0: a fixed share per block)
WALL_GRIDS = (0, 2)                 # blocks per SM of the separate wall kernel (0: as many as fit)

FORM_NAMES = {1: "single_launch", 2: "direct", 3: "two_launch", 4: "dedicated_wall_blocks", 5: "interleaved",
              6: "wall_warps"}

SMEM_LIMIT = 200 * 1024
SINGLE_MARGIN = 0.02       # relative margin by which the single-launch form must win
AGREE = {"f32": 1e-6, "f64": 1e-13}


def cache_path() -> str:
    return os.environ.get("WMIBM_TUNE_CACHE", DEFAULT_CACHE)


def key_of(handle) -> str:
    import torch
    name = torch.cuda.get_device_name(handle.device)
    nx, ny, nz = handle.grid[:3]
    return f"{name}|{handle.dtype}|{handle.vel_dtype}|{nx}x{ny}x{nz}"


def batch_key_of(batch) -> str:
    """GPU, precision and the members' grid sizes in member order."""
    import torch
    h0 = batch.handles[0]
    name = torch.cuda.get_device_name(h0.device)
    grids = ",".join("x".join(str(int(x)) for x in h.grid[:3]) for h in batch.handles)
    digest = hashlib.sha256(grids.encode()).hexdigest()[:16]
    return f"batch|{name}|{h0.dtype}|{h0.vel_dtype}|{len(batch.handles)}|{digest}"


def ring_bytes(rows, stages, nx, es):
    """Shared memory of the stencil's stage rings: `stages` half-A slots of 3 rows + 4
    rows of nx elements and stages + 1 half-B slots of 3 rows + 2."""
    return (stages * (3 * rows + 4) + (stages + 1) * (3 * rows + 2)) * nx * es


def candidates(handle):
    nx, ny, nz = (int(x) for x in handle.grid[:3])
    es = 8 if handle.dtype == "f64" else 4
    vec = 16 // es
    if nx % vec != 0:
        return [dict(force_path=2)]
    out = []
    for rows, stages, cons in itertools.product(ROWS, STAGES, CONSUMERS):
        if ny % rows or ny < rows + 2:
            continue
        if ring_bytes(rows, stages, nx, es) + 256 > SMEM_LIMIT:
            continue
        # one cooperative launch (wall share in every block, dedicated wall blocks,
        # or interleaved wall stages), or the wall kernel followed by the stencil
        out.append(dict(force_path=1, rows=rows, stages=stages, consumer_warps=cons))
        out.append(dict(force_path=4, rows=rows, stages=stages, consumer_warps=cons))
        for per in WALL_CHUNK_PER_THREAD:
            c = dict(force_path=5, rows=rows, stages=stages, consumer_warps=cons)
            if per:
                c["wall_chunk"] = per * 32 * cons
            out.append(c)
        for dyn in DYN_CHUNKS:
            for ww in WALL_WARPS_IN_BLOCK:
                if 1 + cons + ww <= 16:
                    out.append(dict(force_path=6, rows=rows, stages=stages, consumer_warps=cons, wall_warps=ww,
                                    dyn_chunk=dyn))
            for wall in WALL_WARPS:
                for wg in WALL_GRIDS:
                    c = dict(force_path=3, rows=rows, stages=stages, consumer_warps=cons, wall_warps=wall,
                             dyn_chunk=dyn)
                    if wg:
                        c["wall_grid"] = wg
                    out.append(c)
    return out


def batch_candidates(batch):
    h0 = batch.handles[0]
    es = 8 if h0.dtype == "f64" else 4
    max_nx = max(int(h.grid[0]) for h in batch.handles)
    out = []
    for rows, stages, cons in itertools.product((2, 4), (2, 3, 4), (2, 3, 4, 6)):
        # the widest members take `rows` rows per strip; narrower ones more, at about
        # the same stage bytes
        if ring_bytes(rows, stages, max_nx, es) + 256 > SMEM_LIMIT:
            continue
        out.append(dict(force_path=5, rows=rows, stages=stages, consumer_warps=cons))
        for dyn in DYN_CHUNKS:
            out.append(dict(force_path=3, rows=rows, stages=stages, consumer_warps=cons, dyn_chunk=dyn))
            for ww in (1, 2, 3):
                out.append(dict(force_path=6, rows=rows, stages=stages, consumer_warps=cons, wall_warps=ww,
                                dyn_chunk=dyn))
    return out


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class _Flush:
    """256 MiB write (evicts the L2), then a 256 MiB read of another buffer (writes
    the dirty lines back before the timed call)."""

    def __init__(self, device):
        import torch
        self.w = torch.empty(64 << 20, dtype=torch.float32, device=device)
        self.r = torch.ones(64 << 20, dtype=torch.float32, device=device)
        self.acc = torch.zeros((), dtype=torch.float32, device=device)

    def zero_(self):
        import torch
        self.w.zero_()
        torch.sum(self.r, dim=(0,), out=self.acc)


def _median_ms(fn, reps, flush):
    import torch
    for _ in range(2):
        fn()
    times = []
    for _ in range(reps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def time_config(handle, fields, tuning, reps, flush):
    u, v, w, tau, f, stats = fields
    handle.set_tuning(**tuning)
    return _median_ms(lambda: handle.wall_stress_force(u, v, w, tau, f, stats), reps, flush)


def _normwise(a, ref):
    """max |a - ref| / max |ref| over the arrays of two lists of tensors."""
    import torch
    num = max(float(torch.max(torch.abs(x.double() - r.double()))) for x, r in zip(a, ref))
    den = max(float(torch.max(torch.abs(r.double()))) for r in ref)
    return num / den if den > 0 else num


def _forcing_of(run, f_lists):
    """Runs `run()` once and returns copies of every forcing tensor it wrote."""
    import torch
    run()
    torch.cuda.synchronize()
    return [t.clone() for fl in f_lists for t in fl]


def _pick(ranked, check):
    """The first shape of `ranked` (fastest first) whose result agrees with the
    default shape's; returns (ms, tuning, rejected shapes)."""
    rejected = []
    for ms, cand in ranked:
        err = check(cand)
        if err is None:
            continue
        if err <= AGREE["f64" if check.f64 else "f32"]:
            return ms, cand, rejected
        rejected.append({"tuning": cand, "normwise": err})
    return None, None, rejected


def tune(handle, fields, reps: int = 9, use_cache: bool = True, budget_s: float = 60.0,
         verbose: bool = False) -> dict:
    """Finds, applies and caches the fastest tile shape for `handle`.

    fields = (u, v, w, tau[6], f[3], stats) device tensors of the handle's shape;
    the timed call rewrites the band and solid stresses, which does not change
    the work it does.  Returns {"tuning": ..., "ms": ..., "tried": n, "forms_ms":
    fastest time per form, "agreement": normwise difference of the kept shape's
    forcing from the default shape's}."""
    path = cache_path()
    key = key_of(handle)
    cache = _load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        handle.set_tuning(**cache[key]["tuning"])
        return dict(cache[key], cached=True)
    u, v, w, tau, f, stats = fields
    flush = _Flush(handle.device)
    timed = []
    best_form = {}                          # fastest (ms, tuning) per form
    tried = 0
    t_start = time.perf_counter()
    for cand in candidates(handle):
        if time.perf_counter() - t_start > budget_s:
            break
        try:
            ms = time_config(handle, fields, cand, reps, flush)
        except Exception:
            continue
        tried += 1
        if verbose:
            print(f"  {ms * 1e3:8.1f} us  {cand}")
        timed.append((ms, cand))
        form = FORM_NAMES[cand.get("force_path", 1)]
        if form not in best_form or ms < best_form[form][0]:
            best_form[form] = (ms, cand)
    if not timed:
        handle.set_tuning()
        return {"tuning": {}, "ms": None, "tried": tried}
    # a single launch must beat the two-launch form by more than SINGLE_MARGIN to be chosen: within that the two
    # forms are a tie, and the two-launch form keeps each kernel measurable against its own roofline
    two = best_form.get("two_launch")

    def rank(item):
        ms, cand = item
        if two is not None and cand.get("force_path") != 3 and ms > (1.0 - SINGLE_MARGIN) * two[0]:
            return (1, ms)
        return (0, ms)

    ranked = sorted(timed, key=rank)
    handle.set_tuning()
    ref = _forcing_of(lambda: handle.wall_stress_force(u, v, w, tau, f, stats), [f])

    def check(cand):
        try:
            handle.set_tuning(**cand)
            got = _forcing_of(lambda: handle.wall_stress_force(u, v, w, tau, f, stats), [f])
        except Exception:
            return None
        return _normwise(got, ref)

    check.f64 = handle.dtype == "f64"
    ms, cand, rejected = _pick(ranked, check)
    if cand is None:
        handle.set_tuning()
        return {"tuning": {}, "ms": None, "tried": tried, "rejected": rejected}
    handle.set_tuning(**cand)
    agreement = _normwise(_forcing_of(lambda: handle.wall_stress_force(u, v, w, tau, f, stats), [f]), ref)
    result = {"tuning": cand, "ms": ms, "tried": tried, "forms_ms": {k: v[0] for k, v in best_form.items()},
              "agreement": agreement, "rejected": rejected}
    if use_cache:
        cache = _load_cache(path)
        cache[key] = result
        _save_cache(path, cache)
    return dict(result, cached=False)


def tune_batch(batch, stats=None, reps: int = 7, use_cache: bool = True, budget_s: float = 90.0,
               verbose: bool = False) -> dict:
    """Finds, applies and caches the fastest form and tile shape of `batch`
    (whose fields must be set) for wmibm_batch_wall_stress_force.  Returns
    {"tuning", "ms", "tried", "forms_ms", "agreement", "rejected"}."""
    path = cache_path()
    key = batch_key_of(batch)
    cache = _load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        batch.set_tuning(**cache[key]["tuning"])
        return dict(cache[key], cached=True)
    f_lists = [fl[4] for fl in batch._keep]
    flush = _Flush(batch.handles[0].device)
    timed = []
    best_form = {}
    tried = 0
    t_start = time.perf_counter()
    for cand in batch_candidates(batch):
        if time.perf_counter() - t_start > budget_s:
            break
        try:
            batch.set_tuning(**cand)
            ms = _median_ms(lambda: batch.wall_stress_force(stats), reps, flush)
        except Exception:
            continue
        tried += 1
        if verbose:
            print(f"  {ms * 1e3:8.1f} us  {cand}")
        timed.append((ms, cand))
        form = FORM_NAMES[cand["force_path"]]
        if form not in best_form or ms < best_form[form][0]:
            best_form[form] = (ms, cand)
    if not timed:
        batch.set_tuning()
        return {"tuning": {}, "ms": None, "tried": tried}
    ranked = sorted(timed, key=lambda t: t[0])
    batch.set_tuning()
    ref = _forcing_of(lambda: batch.wall_stress_force(stats), f_lists)

    def check(cand):
        try:
            batch.set_tuning(**cand)
            got = _forcing_of(lambda: batch.wall_stress_force(stats), f_lists)
        except Exception:
            return None
        return _normwise(got, ref)

    check.f64 = batch.handles[0].dtype == "f64"
    ms, cand, rejected = _pick(ranked, check)
    if cand is None:
        batch.set_tuning()
        return {"tuning": {}, "ms": None, "tried": tried, "rejected": rejected}
    batch.set_tuning(**cand)
    agreement = _normwise(_forcing_of(lambda: batch.wall_stress_force(stats), f_lists), ref)
    result = {"tuning": cand, "ms": ms, "tried": tried, "forms_ms": {k: v[0] for k, v in best_form.items()},
              "agreement": agreement, "rejected": rejected}
    if use_cache:
        cache = _load_cache(path)
        cache[key] = result
        _save_cache(path, cache)
    return dict(result, cached=False)
