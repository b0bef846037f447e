"""Failure paths on the GPU, caused on the host or by a bounded wait that runs out
(nothing here faults, traps or hangs a GPU):

- an injected allocation failure (WMIBM_FAULT=alloc:N) at every allocation of
  wmibm_init, of wmibm_batch_create and of the adjoint map: the call returns
  ENOMEM and gives back all the device memory it took;
- a single-launch stage whose blocks never count themselves as done with the
  wall model (WMIBM_FAULT=hold_release, with WMIBM_WAIT_LIMIT_NS of 1 ms): its
  bounded waits run out, the kernel returns, wmibm_device_status reports
  ETIMEOUT, and the device stays usable: a handle made without the hook matches
  the oracle afterwards.
"""
import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import TOL, assert_stats_close, gpu_fused, normwise, oracle_step, to_dev

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


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _sweep(fn, wm, monkeypatch, limit=80):
    """Calls fn() with the N-th allocation failing for N = 1, 2, ... until it goes
    through; every failing call must raise ENOMEM and leave the free device memory
    where it was.  Returns the number of allocations fn makes."""
    for n in range(1, limit):
        monkeypatch.setenv("WMIBM_FAULT", f"alloc:{n}")
        before = _free_bytes()
        try:
            obj = fn()
        except wm.WmibmError as e:
            assert e.status == wm.ENOMEM, (n, str(e))
            assert _free_bytes() == before, (n, "device memory not given back")
            continue
        monkeypatch.delenv("WMIBM_FAULT")
        obj.close()
        return n - 1
    raise AssertionError("the call never went through")


def test_init_allocation_failures(wm, monkeypatch):
    case = inputs.cubes(shape=(64, 32, 24))          # power-of-two plane: the spectral tables too
    wm.Handle.from_case(case).close()                # the library's kernels are loaded before the sweep
    n = _sweep(lambda: wm.Handle.from_case(case), wm, monkeypatch)
    assert n >= 15                                   # every list, record, run and scratch allocation was hit


def test_batch_create_allocation_failures(wm, monkeypatch):
    cases = [inputs.ensemble_member(m, shape=(64, 32, 24)) for m in range(3)]
    handles = [wm.Handle.from_case(c) for c in cases]
    n = _sweep(lambda: wm.Batch(handles), wm, monkeypatch)
    assert n >= 5


def test_adjoint_map_allocation_failure(wm, monkeypatch):
    """The adjoint map's allocations (made at the first wmibm_set_log_z0) fail with
    ENOMEM, free what they took, and a later call builds the map."""
    case, _ = inputs.adjoint_case(shape=(64, 32, 24), dtype="f32")
    s = to_dev(np.log(case.z0), "f32")
    # the count armed at init goes on after it: the smallest N with which init goes
    # through fails the first allocation after init, the adjoint map's
    probe = 0
    for k in range(1, 80):
        monkeypatch.setenv("WMIBM_FAULT", f"alloc:{k}")
        try:
            h = wm.Handle.from_case(case)
        except wm.WmibmError:
            continue
        probe = k                                     # init made k - 1 allocations; the k-th is the map's first
        break
    assert probe > 0
    before = _free_bytes()
    with pytest.raises(wm.WmibmError) as e:
        h.set_log_z0(s)
    assert e.value.status == wm.ENOMEM
    assert _free_bytes() == before
    monkeypatch.delenv("WMIBM_FAULT")
    h.set_log_z0(s)                                   # builds the map now
    torch.cuda.synchronize()
    h.close()


@pytest.mark.parametrize("form", [1, 4, 5, 6])
def test_single_launch_wait_runs_out(wm, oracle_mod, monkeypatch, form):
    case = inputs.cubes(shape=(96, 48, 40))
    monkeypatch.setenv("WMIBM_FAULT", "hold_release")
    monkeypatch.setenv("WMIBM_WAIT_LIMIT_NS", "1000000")
    h = wm.Handle.from_case(case)
    monkeypatch.delenv("WMIBM_FAULT")
    monkeypatch.delenv("WMIBM_WAIT_LIMIT_NS")
    h.set_tuning(force_path=form)
    gpu_fused(h, case, "f32")                         # returns: every wait is bounded
    assert h.device_status() == wm.ETIMEOUT
    assert h.device_status() == wm.OK                 # reading clears the word
    h.close()
    # the device is usable, and a handle without the hook is right
    h2 = wm.Handle.from_case(case)
    h2.set_tuning(force_path=form)
    tau_g, f_g, st_g = gpu_fused(h2, case, "f32")
    tau_o, f_o, st_o = oracle_step(oracle_mod, case)
    for c in range(3):
        assert normwise(f_g[c], f_o[c])[0] <= TOL["f32"]
    for k in inputs.TAU_NAMES:
        assert normwise(tau_g[k], tau_o[k])[0] <= TOL["f32"]
    assert_stats_close(st_g, st_o, "f32")
    assert h2.device_status() == wm.OK
    h2.close()


def test_batch_single_launch_wait_runs_out(wm, monkeypatch):
    cases = [inputs.ensemble_member(m, shape=(64, 32, 24)) for m in range(3)]
    handles = [wm.Handle.from_case(c) for c in cases]
    monkeypatch.setenv("WMIBM_FAULT", "hold_release")
    monkeypatch.setenv("WMIBM_WAIT_LIMIT_NS", "1000000")
    batch = wm.Batch(handles)
    monkeypatch.delenv("WMIBM_FAULT")
    monkeypatch.delenv("WMIBM_WAIT_LIMIT_NS")
    batch.set_tuning(force_path=6)
    d = lambda a: to_dev(a, "f32")
    fields = [(d(c.u), d(c.v), d(c.w), [d(c.tau[k]) for k in inputs.TAU_NAMES],
               [torch.empty(c.shape, dtype=torch.float32, device="cuda") for _ in range(3)]) for c in cases]
    batch.set_fields(fields)
    batch.wall_stress_force(batch.new_stats())
    torch.cuda.synchronize()
    assert batch.device_status() == wm.ETIMEOUT
    assert batch.device_status() == wm.OK
    assert torch.ones(1024, device="cuda").sum().item() == 1024.0
    batch.close()
