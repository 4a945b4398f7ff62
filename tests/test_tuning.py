"""Autotuner: shape classes, the JSON cache and applying a cached tuning (host only), and one
short tuning run on the GPU whose bits must not change."""
import numpy as np
import pytest

from paper_2306_04316_gb300 import tuning


def test_shape_class_is_coarse_and_deterministic():
    a = tuning.shape_class(1_000_000, 7_000_000, 16_000_000, False)
    assert a == tuning.shape_class(1_000_001, 7_000_100, 16_000_050, False)
    assert a != tuning.shape_class(64, 13_000_000, 4_000_000, False)
    assert tuning.shape_class(1, 1024, 101_000, True).startswith("dense-")


def test_cache_round_trip_and_apply(tmp_path, monkeypatch):
    from paper_2306_04316_gb300 import api, build
    build.build_library()
    monkeypatch.setenv("PIP_TUNING_CACHE", str(tmp_path / "t.json"))
    before = api.pip_get_tuning()
    try:
        cls = tuning.shape_class(64, 13_000_000, 4_000_000, False)
        tuning._store_cache(tuning.cache_path(), {tuning._key("GB300", cls): {"tuning": [1024, 4, 3], "ms": 1.0}})
        assert tuning.apply_cached(64, 13_000_000, 4_000_000, False, "GB300") == (1024, 4, 3)
        assert api.pip_get_tuning() == (1024, 4, 3)
        assert tuning.apply_cached(5, 50, 50, True, "GB300") is None
    finally:
        api.pip_set_tuning(*before)


@pytest.mark.gpu
def test_autotune_on_gpu(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_04316_gb300 import api, workloads as W
    monkeypatch.setenv("PIP_TUNING_CACHE", str(tmp_path / "t.json"))
    before = api.pip_get_tuning()
    try:
        w = W.fractal(seed=91, n_polys=4, m_lo=3000, m_hi=6000, n_points=40_000, cell=300_000, grid=2)
        d = api.to_device(w)
        ref = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], d["cand_offsets"], d["cand_ids"],
                               n_cands=w.n_bits).clone()
        grid = [(1024, 1, 2), (2048, 2, 4), (4096, 4, 3)]
        best, times = tuning.autotune(d["points"], d["poly_offsets"], d["verts"], d["cand_offsets"], d["cand_ids"],
                                      n_cands=w.n_bits, grid=grid, reps=2)
        assert best in grid and set(times) == set(grid) and api.pip_get_tuning() == best
        got = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], d["cand_offsets"], d["cand_ids"],
                               n_cands=w.n_bits)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        name = torch.cuda.get_device_name(0)
        assert tuning.apply_cached(w.n_polys, w.verts.shape[0], w.n_bits, False, name) == best
    finally:
        api.pip_set_tuning(*before)


@pytest.mark.gpu
def test_autotune_small_on_gpu(tmp_path, monkeypatch):
    """The small-polygon kernel's tuner: every shape of its grid timed, the fastest applied and
    cached, and the bits unchanged."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_04316_gb300 import api, workloads as W
    monkeypatch.setenv("PIP_TUNING_CACHE", str(tmp_path / "t.json"))
    before = api.pip_get_small_tuning()
    try:
        w = W.footprints(seed=93, n_polys=20_000, pts_per_poly=16)
        d = api.to_device(w)
        ref = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], d["cand_offsets"], d["cand_ids"],
                               n_cands=w.n_bits).clone()
        best, times = tuning.autotune_small(d["points"], d["poly_offsets"], d["verts"], d["cand_offsets"],
                                            d["cand_ids"], n_cands=w.n_bits, reps=2)
        assert best in tuning.SMALL_GRID and set(times) == set(tuning.SMALL_GRID)
        assert api.pip_get_small_tuning() == best
        got = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], d["cand_offsets"], d["cand_ids"],
                               n_cands=w.n_bits)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        api.pip_set_small_tuning(*before)
        tuning.apply_cached(w.n_polys, w.verts.shape[0], w.n_bits, False, torch.cuda.get_device_name(0))
        assert api.pip_get_small_tuning() == best
    finally:
        api.pip_set_small_tuning(*before)
