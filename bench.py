"""Benchmark of the wall-modeled IBM stress stage on GB300.

One step = wall stress (band wall model + solid zeroing) -> force (f = -div tau)
-> body mask, i.e. one pass of the whole per-step stage, through the C ABI.
Default workload: the 4 x 4 wall-mounted cube array on a 256 x 128 x 128 grid in
FP32 (4.19 M nodes).  The metric is nodes per second (Gpts/s); the roofline
figure is the force kernel's achieved HBM bandwidth over the measured copy peak.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this project)
on the same workload.  Under torchrun with N > 1 every rank runs its own
replica of the workload on its own GPU (independent problems, no collective on
the data path; weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IBM wall-stress+forcing throughput (Gpts/s)"
UNIT = "Gpts/s"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cubes", choices=["cubes", "hill", "ridge"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--vel-dtype", default=None, choices=[None, "bf16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic(kernel_file, workload, dtype):
    """DRAM bytes per launch of the force kernel from the committed ncu summary,
    if that summary was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"force_{workload}_{dtype}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    src = open(kernel_file, "rb").read()
    digest = hashlib.sha256(src).hexdigest()[:16]
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != digest:
        return None
    return float(m_bytes.group(1))


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while the GPU is busy."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_case(args):
    from paper_2006_03343_gb300 import inputs
    return inputs.make(args.workload, dtype=args.dtype)


def workload_config(args, case):
    nx, ny, nz = case.grid[:3]
    return {"workload": f"{case.name} {nx}x{ny}x{nz}", "nodes": case.npoints, "dtype": args.dtype,
            "vel_storage": args.vel_dtype or args.dtype, "phi_c": "1.5 dz", "z0": "per-cell" if not np.isscalar(
                case.z0) else case.z0, "l2": "flushed between steps (256 MiB write, outside the timed events)"}


# --------------------------------------------------------------------------- #
# CPU oracle timing (reference arm and cpu_baseline)
# --------------------------------------------------------------------------- #
def oracle_time(case, seconds):
    """Times the oracle's wall_stress + force + mask on full copies of the workload
    for about `seconds` (at least one pass). Returns (Gpts/s, passes, threads)."""
    import oracle
    oracle.build()
    tau = {k: v.copy() for k, v in case.tau.items()}
    u, v, w = case.u.copy(), case.v.copy(), case.w.copy()
    passes = 0
    t0 = time.perf_counter()
    while True:
        oracle.wall_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b, u, v, w, tau)
        oracle.force(case.grid, tau)
        oracle.mask(case.grid, case.phi_uv, case.phi_w, u, v, w)
        passes += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return passes * case.npoints / el / 1e9, passes, oracle.openmp_threads(), el


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    case = make_case(args)
    for _ in range(max(args.warmup, 0)):
        pass
    per_step = []
    import oracle
    oracle.build()
    tau = {k: v.copy() for k, v in case.tau.items()}
    u, v, w = case.u.copy(), case.v.copy(), case.w.copy()
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.wall_stress(case.grid, case.phi_uv, case.phi_w, case.z0, case.phi_c, case.phi_b, u, v, w, tau)
        oracle.force(case.grid, tau)
        oracle.mask(case.grid, case.phi_uv, case.phi_w, u, v, w)
        if s >= args.warmup:
            per_step.append(time.perf_counter() - t0)
    total = sum(per_step)
    value = args.steps * case.npoints / total / 1e9
    threads = oracle.openmp_threads()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, case),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} full passes of the workload (FP64 CPU oracle)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- #
# GPU arm
# --------------------------------------------------------------------------- #
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2006_03343_gb300 import build, inputs, wmibm
    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    case = make_case(args)
    h = wmibm.Handle.from_case(case, dtype=args.dtype, vel_dtype=args.vel_dtype)
    tdt = torch.float64 if args.dtype == "f64" else torch.float32
    vdt = torch.bfloat16 if args.vel_dtype == "bf16" else tdt

    def dev_t(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dt)

    u, v, w = (dev_t(x, vdt) for x in (case.u, case.v, case.w))
    tau = [dev_t(case.tau[k], tdt) for k in inputs.TAU_NAMES]
    f = [torch.empty(case.shape, dtype=tdt, device=dev) for _ in range(3)]
    stats = h.new_stats()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        h.wall_stress(u, v, w, tau, stats)
        if evs is not None:
            evs[1].record(stream)
        h.force(tau, f)
        if evs is not None:
            evs[2].record(stream)
        h.mask(u, v, w)
        if evs is not None:
            evs[3].record(stream)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    # keep the GPU busy ~1 s before the timed region so the clock sampler sees load
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < 1.0:
        for _ in range(20):
            flush.zero_()
            step()
        torch.cuda.synchronize()

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.zero_()
        step(events[s])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None

    step_ms = [e[0].elapsed_time(e[3]) for e in events]
    ws_ms = [e[0].elapsed_time(e[1]) for e in events]
    force_ms = [e[1].elapsed_time(e[2]) for e in events]
    mask_ms = [e[2].elapsed_time(e[3]) for e in events]
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps * case.npoints / (total_ms * 1e-3) / 1e9

    # roofline of the dominant kernel (force)
    force_bytes = h.traffic_bytes(1)
    force_avg_s = float(np.mean(force_ms)) * 1e-3
    peak, peak_kind = measured_peak()
    achieved = force_bytes / force_avg_s / 1e9
    kernel_file = os.path.join(ROOT, "paper_2006_03343_gb300", "csrc", "force.cu")
    traffic = profiled_traffic(kernel_file, args.workload, args.dtype)

    # end to end through the public API: pinned host inputs in, forcing out
    e2e = None
    if not args.no_e2e:
        host_in = [torch.from_numpy(np.ascontiguousarray(x)).to(vdt).pin_memory() for x in (case.u, case.v, case.w)]
        host_tau = [torch.from_numpy(case.tau[k]).to(tdt).pin_memory() for k in inputs.TAU_NAMES]
        host_f = [torch.empty(case.shape, dtype=tdt).pin_memory() for _ in range(3)]
        h2d = sum(t.numel() * t.element_size() for t in host_in + host_tau)
        d2h = sum(t.numel() * t.element_size() for t in host_f) + stats.numel() * 8
        host_stats = torch.empty(10, dtype=torch.float64).pin_memory()

        def e2e_step():
            for d, s_ in zip((u, v, w), host_in):
                d.copy_(s_, non_blocking=True)
            for d, s_ in zip(tau, host_tau):
                d.copy_(s_, non_blocking=True)
            h.step(u, v, w, tau, f, None, 0.0, stats)
            for d, s_ in zip(host_f, f):
                d.copy_(s_, non_blocking=True)
            host_stats.copy_(stats, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([el], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * args.steps * case.npoints / el / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        gpts, passes, threads, el = oracle_time(case, args.cpu_seconds)
        cpu = {"value": gpts, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{passes} full passes of the workload ({el:.1f} s, FP64 CPU oracle)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
                "config": workload_config(args, case),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "kernel": "k_force",
                             "peak_source": f"{peak_kind} hbm_gbs (burst copy)",
                             "algorithmic_bytes_per_launch": force_bytes},
                "kernels_ms": {"wall_stress": float(np.mean(ws_ms)), "force": float(np.mean(force_ms)),
                               "mask": float(np.mean(mask_ms))},
                "step_bytes": h.traffic_bytes(0) + force_bytes + h.traffic_bytes(2),
                "step_gbs": (h.traffic_bytes(0) + force_bytes + h.traffic_bytes(2)) / (total_ms / args.steps * 1e-3) / 1e9,
                "gpu_launches": 3 * args.steps,
                "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line))
    h.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
