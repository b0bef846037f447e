"""Host logic of the autotuner, on the CPU: the candidate shapes it times (every
one fits the stencil's shared-memory rings and the grid's strips), the choice of
the fastest shape whose forcing agrees with the default shape's (a shape that
disagrees is rejected and reported, one that fails to run is skipped), and the
cache file (written atomically, unreadable contents treated as empty)."""
import types

import pytest

from paper_2006_03343_gb300 import autotune


def _handle(nx, ny, nz, dtype="f32"):
    return types.SimpleNamespace(grid=(nx, ny, nz, 1.0, 1.0, 1.0), dtype=dtype)


@pytest.mark.parametrize("grid,dtype", [((256, 128, 128), "f32"), ((512, 256, 256), "f32"),
                                        ((256, 128, 128), "f64"), ((96, 48, 40), "f32"), ((64, 6, 10), "f64")])
def test_candidates_fit_and_cover_every_form(grid, dtype):
    nx, ny, nz = grid
    es = 8 if dtype == "f64" else 4
    cands = autotune.candidates(_handle(nx, ny, nz, dtype))
    assert cands
    forms = {c["force_path"] for c in cands}
    assert forms == {1, 3, 4, 5, 6}
    for c in cands:
        assert ny % c["rows"] == 0 and ny >= c["rows"] + 2, c
        assert autotune.ring_bytes(c["rows"], c["stages"], nx, es) + 256 <= autotune.SMEM_LIMIT, c
        if c["force_path"] == 6:
            assert 1 + c["consumer_warps"] + c["wall_warps"] <= 16, c
        assert c["force_path"] in autotune.FORM_NAMES


def test_candidates_without_vector_rows_take_the_direct_kernel():
    # rows of 30 floats are no whole number of 16-byte vectors: only the direct-load kernel applies
    assert autotune.candidates(_handle(30, 16, 8)) == [dict(force_path=2)]
    assert autotune.candidates(_handle(7, 16, 8, "f64")) == [dict(force_path=2)]


def test_batch_candidates_fit_the_widest_member():
    batch = types.SimpleNamespace(handles=[_handle(64, 64, 64), _handle(256, 128, 64), _handle(192, 96, 96)])
    cands = autotune.batch_candidates(batch)
    assert {c["force_path"] for c in cands} == {3, 5, 6}
    for c in cands:
        assert autotune.ring_bytes(c["rows"], c["stages"], 256, 4) + 256 <= autotune.SMEM_LIMIT, c


def _check(errors, f64=False):
    def check(cand):
        return errors[cand["id"]]
    check.f64 = f64
    return check


def test_pick_keeps_the_fastest_agreeing_shape():
    ranked = [(1.0, {"id": 0}), (1.1, {"id": 1}), (1.2, {"id": 2}), (1.3, {"id": 3})]
    # 0 disagrees, 1 fails to run, 2 agrees
    ms, cand, rejected = autotune._pick(ranked, _check({0: 1e-3, 1: None, 2: 5e-7, 3: 0.0}))
    assert (ms, cand) == (1.2, {"id": 2})
    assert rejected == [{"tuning": {"id": 0}, "normwise": 1e-3}]


def test_pick_uses_the_precision_tolerance():
    ranked = [(1.0, {"id": 0}), (2.0, {"id": 1})]
    err = autotune.AGREE["f32"] / 2          # within FP32's tolerance, far outside FP64's
    ms, cand, rejected = autotune._pick(ranked, _check({0: err, 1: 0.0}))
    assert cand == {"id": 0} and not rejected
    ms, cand, rejected = autotune._pick(ranked, _check({0: err, 1: 0.0}, f64=True))
    assert cand == {"id": 1} and rejected[0]["tuning"] == {"id": 0}


def test_pick_with_no_agreeing_shape_returns_none():
    ranked = [(1.0, {"id": 0}), (2.0, {"id": 1})]
    ms, cand, rejected = autotune._pick(ranked, _check({0: 1.0, 1: None}))
    assert ms is None and cand is None and len(rejected) == 1


def test_cache_round_trip_and_unreadable_file(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    assert autotune._load_cache(path) == {}
    data = {"k": {"tuning": {"rows": 4}, "ms": 0.5}}
    autotune._save_cache(path, data)
    assert autotune._load_cache(path) == data
    assert not [p for p in (tmp_path / "sub").iterdir() if ".tmp" in p.name]   # no temporary left behind
    with open(path, "w") as f:
        f.write("{not json")
    assert autotune._load_cache(path) == {}


def test_cache_path_follows_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("WMIBM_TUNE_CACHE", str(tmp_path / "c.json"))
    assert autotune.cache_path() == str(tmp_path / "c.json")
    monkeypatch.delenv("WMIBM_TUNE_CACHE")
    assert autotune.cache_path() == autotune.DEFAULT_CACHE
