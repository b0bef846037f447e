"""The wall-stress entry point that allocates no device memory.

It exists for callers that cannot allocate device memory when they call (for
example while a CUDA graph is being captured, or inside a host framework that
owns the device memory pool): its reduction scratch is a static device array.
This file is collected last on purpose, so that a run that stops at the first
failure has run every other test; it must also pass alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2006_03343_gb300 import inputs

from parity_util import STATS_TOL, normwise, to_dev, to_host

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


def _fields(case, dtype):
    u, v, w = (to_dev(x, dtype) for x in (case.u, case.v, case.w))
    tau = [to_dev(case.tau[k], dtype) for k in inputs.TAU_NAMES]
    return u, v, w, tau


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_wall_stress_twice(wm, dtype):
    """Two calls in a row through the C ABI give the stresses and band statistics
    of wmibm_wall_stress (the static scratch is reused and re-armed)."""
    case = inputs.hill(shape=(128, 64, 48))
    h = wm.Handle.from_case(case, dtype=dtype)
    u, v, w, tau_ref = _fields(case, dtype)
    stats_ref = h.new_stats()
    h.wall_stress(u, v, w, tau_ref, stats_ref)
    torch.cuda.synchronize()
    ref_tau = [to_host(t) for t in tau_ref]
    ref_stats = h.parse_stats(stats_ref)
    tol = 1e-12 if dtype == "f64" else 1e-6
    for call in range(2):
        _, _, _, tau = _fields(case, dtype)
        stats = h.new_stats()
        L = wm.load()
        tau_ptrs = (ctypes.c_void_p * 6)(*[t.data_ptr() for t in tau])
        st = L.wmibm_wall_stress_noalloc(h.raw, u.data_ptr(), v.data_ptr(), w.data_ptr(), tau_ptrs,
                                         stats.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == wm.OK, L.wmibm_last_error(h.raw)
        torch.cuda.synchronize()
        for got, ref in zip(tau, ref_tau):
            assert normwise(to_host(got), ref)[0] <= tol, call
        got_stats = h.parse_stats(stats)
        for b in range(2):
            assert got_stats[b]["count"] == ref_stats[b]["count"]
            for name in ("sum_tw", "sum_tw2", "min_tw", "max_ur"):
                assert got_stats[b][name] == pytest.approx(ref_stats[b][name], rel=STATS_TOL[dtype], abs=1e-300)
    assert h.device_status() == wm.OK


def test_noalloc_binding_and_empty_band(wm):
    """The binding method, and a terrain with no band at all (statistics zero)."""
    case = inputs.flat((16, 8, 9), wall_height=-0.5, sigma=0.3, seed=2)
    h = wm.Handle.from_case(case, dtype="f32")
    u, v, w, tau = _fields(case, "f32")
    stats = h.new_stats()
    h.wall_stress_noalloc(u, v, w, tau, stats)
    torch.cuda.synchronize()
    s = h.parse_stats(stats)
    assert s[0]["count"] == 0 and s[1]["count"] == 0 and s[0]["sum_tw"] == 0.0
    for t, name in zip(tau, inputs.TAU_NAMES):
        assert np.array_equal(to_host(t), np.float32(case.tau[name]).astype(np.float64))
