"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/wmibm.h declares, and rejects bad arguments on the host
(no GPU needed: validation happens before any CUDA call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2006_03343_gb300 import build as wbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    wbuild.build()
    from paper_2006_03343_gb300 import wmibm
    return wmibm.load()


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(wmibm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_api():
    names = _declared_functions()
    for required in ("wmibm_init", "wmibm_wall_stress", "wmibm_force", "wmibm_mask", "wmibm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(_declared_functions()):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_lists_match_header():
    from paper_2006_03343_gb300 import wmibm
    assert set(wmibm.EXPORTED) <= _declared_functions()


def test_status_strings(lib):
    assert lib.wmibm_status_string(0) == b"ok"
    assert lib.wmibm_status_string(1) == b"invalid argument"
    assert lib.wmibm_status_string(99) == b"unknown status"


def _init(lib, grid, phi_uv, phi_w, z0, phi_c, opts=None, z0_field=0):
    from paper_2006_03343_gb300 import wmibm
    h = ctypes.c_void_p()
    g = None if grid is None else wmibm.Grid(*grid)
    st = lib.wmibm_init(ctypes.byref(h), None if g is None else ctypes.byref(g),
                        None if phi_uv is None else phi_uv.ctypes.data,
                        None if phi_w is None else phi_w.ctypes.data,
                        None if z0 is None else z0.ctypes.data, z0_field, phi_c,
                        None if opts is None else ctypes.byref(opts), None)
    return st, h, lib.wmibm_last_error(None).decode()


def test_init_rejects_bad_arguments_on_host(lib):
    from paper_2006_03343_gb300 import wmibm
    phi = np.ones((5, 4, 4))
    z0 = np.array([1e-4])
    dz = 1.0 / 4
    ok_grid = (4, 4, 5, 1.0, 1.0, 1.0)
    assert _init(lib, None, phi, phi, z0, 1.5 * dz)[0] == wmibm.EINVAL
    assert _init(lib, (4, 4, 2, 1.0, 1.0, 1.0), phi, phi, z0, 1.5 * dz)[0] == wmibm.EINVAL      # nz < 3
    assert _init(lib, (4, 4, 5, -1.0, 1.0, 1.0), phi, phi, z0, 1.5 * dz)[0] == wmibm.EINVAL     # length
    st, h, msg = _init(lib, ok_grid, phi, phi, np.array([1.0]), 1.5 * dz)                       # z0 >= phi_c
    assert st == wmibm.EINVAL and "z0" in msg and not h.value
    assert _init(lib, ok_grid, phi, phi, z0, 0.5 * dz)[0] == wmibm.EINVAL                       # phi_c < 2 phi_b
    bad = phi.copy()
    bad[2, 1, 1] = np.nan
    st, _, msg = _init(lib, ok_grid, bad, phi, z0, 1.5 * dz)
    assert st == wmibm.EINVAL and "phi" in msg
    o = wmibm.Opts(0.0, 0.0, wmibm.F64, wmibm.BF16)                                            # bf16 needs f32
    assert _init(lib, ok_grid, phi, phi, z0, 1.5 * dz, o)[0] == wmibm.EINVAL
    zf = np.full((5, 4, 4), 1e-4)
    zf[4, 3, 3] = 0.0
    assert _init(lib, ok_grid, phi, phi, zf, 1.5 * dz, None, 1)[0] == wmibm.EINVAL              # z0 field


def test_calls_reject_null_handle(lib):
    from paper_2006_03343_gb300 import wmibm
    tau = (ctypes.c_void_p * 6)()
    assert lib.wmibm_wall_stress(None, None, None, None, tau, None, None) == wmibm.EINVAL
    assert lib.wmibm_force(None, tau, None, None, None, None) == wmibm.EINVAL
    assert lib.wmibm_mask(None, None, None, None, None, 0.0, None) == wmibm.EINVAL
    assert lib.wmibm_list_size(None, 0) == -1
    assert lib.wmibm_traffic_bytes(None, 0) == -1
    lib.wmibm_destroy(None)


def test_later_entry_points_reject_null_arguments(lib):
    """The step, spectral, SGS, adjoint, tuning and batch entry points refuse NULL
    handles and tables on the host, before anything reaches a GPU."""
    from paper_2006_03343_gb300 import wmibm
    tau = (ctypes.c_void_p * 6)()
    three = (ctypes.c_void_p * 3)()
    assert lib.wmibm_step(None, None, None, None, tau, None, None, None, None, 0.0, None, None) == wmibm.EINVAL
    assert lib.wmibm_wall_stress_force(None, None, None, None, tau, None, None, None, None, None) == wmibm.EINVAL
    assert lib.wmibm_force_mask(None, tau, None, None, None, None, None, None, None, 0.0, None) == wmibm.EINVAL
    assert lib.wmibm_wall_stress_noalloc(None, None, None, None, tau, None, None) == wmibm.EINVAL
    assert lib.wmibm_force_spectral(None, tau, None, None, None, None) == wmibm.EINVAL
    assert lib.wmibm_spectral_shape(None, (ctypes.c_int64 * 4)()) == wmibm.EINVAL
    assert lib.wmibm_sgs_wall_terms(None, None, None, None, 0, None, None, None) == wmibm.EINVAL
    assert lib.wmibm_sgs_stress(None, None, None, None, None, None, tau, 0.16, None) == wmibm.EINVAL
    assert lib.wmibm_sgs_force(None, None, None, None, None, None, tau, None, None, None, 0.16, None) == wmibm.EINVAL
    assert lib.wmibm_set_log_z0(None, None, None) == wmibm.EINVAL
    assert lib.wmibm_backward(None, three, three, None, None, None, None, None) == wmibm.EINVAL
    t = wmibm.Tuning()
    assert lib.wmibm_set_tuning(None, ctypes.byref(t)) == wmibm.EINVAL
    assert lib.wmibm_get_tuning(None, ctypes.byref(t)) == wmibm.EINVAL
    out = ctypes.c_void_p()
    assert lib.wmibm_batch_create(ctypes.byref(out), None, 1, None) == wmibm.EINVAL and not out.value
    handles = (ctypes.c_void_p * 1)()
    assert lib.wmibm_batch_create(ctypes.byref(out), handles, 1, None) == wmibm.EINVAL      # NULL member
    assert lib.wmibm_batch_create(ctypes.byref(out), handles, 0, None) == wmibm.EINVAL      # no members
    assert lib.wmibm_batch_step(None, None, None) == wmibm.EINVAL
    assert lib.wmibm_batch_wall_stress_force(None, None, None) == wmibm.EINVAL
    assert lib.wmibm_batch_set_fields(None, None, None) == wmibm.EINVAL
    assert lib.wmibm_batch_traffic_bytes(None, 0) == -1
    assert lib.wmibm_batch_points(None) == -1
    lib.wmibm_batch_destroy(None)


def test_init_rejects_unknown_zclamp_mode(lib):
    from paper_2006_03343_gb300 import wmibm
    phi = np.ones((5, 4, 4))
    o = wmibm.Opts(0.0, 0.0, wmibm.F32, wmibm.F32, 7)
    st, h, msg = _init(lib, (4, 4, 5, 1.0, 1.0, 1.0), phi, phi, np.array([1e-4]), 1.5 / 4, o)
    assert st == wmibm.EINVAL and "zclamp" in msg and not h.value


def test_injected_allocation_failure_before_any_gpu_work(lib, monkeypatch):
    """WMIBM_FAULT=alloc:1 fails the first allocation of wmibm_init (the handle's
    host memory, made before any CUDA call): ENOMEM, no handle, a message; unset,
    the same call gets past it (to the device query, which has no GPU here)."""
    from paper_2006_03343_gb300 import wmibm
    phi = np.ones((5, 4, 4))
    args = ((4, 4, 5, 1.0, 1.0, 1.0), phi, phi, np.array([1e-4]), 1.5 / 4)
    monkeypatch.setenv("WMIBM_FAULT", "alloc:1")
    st, h, msg = _init(lib, *args)
    assert st == wmibm.ENOMEM and not h.value and "allocation" in msg
    monkeypatch.delenv("WMIBM_FAULT")
    st, h, _ = _init(lib, *args)
    assert st != wmibm.ENOMEM
    if st == wmibm.OK:
        lib.wmibm_destroy(h)


def test_struct_layouts_match_the_header(tmp_path):
    """The Python mirrors of the header's structs (ctypes Grid, Opts, Tuning,
    MemberFields and the numpy record of wmibm_band_stats) have the C compiler's
    size and field offsets, so that a field added to the header without its
    mirror, or in another order, fails here rather than corrupting a call."""
    import shutil
    import subprocess
    from paper_2006_03343_gb300 import wmibm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"wmibm_grid": wmibm.Grid, "wmibm_opts": wmibm.Opts, "wmibm_tuning": wmibm.Tuning,
               "wmibm_member_fields": wmibm.MemberFields}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "wmibm.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('    printf("wmibm_band_stats size %zu\\n", sizeof(wmibm_band_stats));')
    for fname in wmibm.STATS_DTYPE.names:
        lines.append(f'    printf("wmibm_band_stats {fname} %zu\\n", offsetof(wmibm_band_stats, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        parts = line.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, cls in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
    assert got[("wmibm_band_stats", "size")] == wmibm.STATS_DTYPE.itemsize
    for fname in wmibm.STATS_DTYPE.names:
        assert got[("wmibm_band_stats", fname)] == wmibm.STATS_DTYPE.fields[fname][1], fname
