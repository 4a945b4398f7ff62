"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads,
exports every function declared in include/pip.h, and rejects bad arguments before it
touches a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_04316_gb300 import build, _lib
    build.build_library()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pip.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(pip_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("pip_classify", "pip_classify_exact", "pip_bin_count", "pip_bin_fill",
                 "pip_set_tuning", "pip_get_stats", "pip_validate", "pip_status_str"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_symbol(lib):
    from paper_2306_04316_gb300 import _lib
    assert sorted(_lib._SIGS) == declared_functions()


def test_status_strings(lib):
    for code in range(-7, 1):
        assert lib.pip_status_str(code).startswith(b"PIP_")
    assert lib.pip_version() >= 100
    assert lib.pip_launch_count() >= 0


def test_argument_checks_return_before_any_device_call(lib):
    from paper_2306_04316_gb300 import _lib
    P = ctypes.c_void_p
    a8 = P(0x1000)          # never dereferenced: every call below fails its host checks
    odd = P(0x1004)
    # negative sizes
    assert lib.pip_classify(a8, -1, a8, a8, 1, None, None, a8, None) == _lib.PIP_ERR_SIZE
    assert lib.pip_classify(a8, 4, a8, a8, -2, None, None, a8, None) == _lib.PIP_ERR_SIZE
    # only one half of the CSR
    assert lib.pip_classify(a8, 4, a8, a8, 1, a8, None, a8, None) == _lib.PIP_ERR_NULL
    assert lib.pip_classify_exact(a8, 4, a8, a8, 1, None, a8, a8, None) == _lib.PIP_ERR_NULL
    # missing arrays
    assert lib.pip_classify(None, 4, a8, a8, 1, None, None, a8, None) == _lib.PIP_ERR_NULL
    assert lib.pip_classify(a8, 4, None, a8, 1, None, None, a8, None) == _lib.PIP_ERR_NULL
    assert lib.pip_classify(a8, 4, a8, a8, 1, None, None, None, None) == _lib.PIP_ERR_NULL
    # int2 arrays must be 8-byte aligned
    assert lib.pip_classify(odd, 4, a8, a8, 1, None, None, a8, None) == _lib.PIP_ERR_ALIGN
    assert lib.pip_classify(a8, 4, a8, odd, 1, None, None, a8, None) == _lib.PIP_ERR_ALIGN
    assert lib.pip_classify(a8, 4, P(0x1002), a8, 1, None, None, a8, None) == _lib.PIP_ERR_ALIGN
    # ids are int32
    assert lib.pip_classify(a8, 2**31, a8, a8, 1, None, None, a8, None) == _lib.PIP_ERR_TOO_LARGE
    # nothing to do: no polygons
    assert lib.pip_classify(a8, 4, a8, a8, 0, None, None, a8, None) == _lib.PIP_OK
    # binning
    assert lib.pip_bin_count(a8, 4, a8, a8, 1, -1, a8, 1 << 30, a8, a8, None) == _lib.PIP_ERR_SIZE
    assert lib.pip_bin_count(a8, 4, a8, a8, 1, 0, a8, 16, a8, a8, None) == _lib.PIP_ERR_WORKSPACE
    assert lib.pip_bin_fill(a8, 4, a8, a8, 1, a8, 1 << 30, a8, a8, -1, None, None) == _lib.PIP_ERR_SIZE
    # validate
    assert lib.pip_validate(a8, 4, a8, a8, 1, 4, None, None, 0, None, None) == _lib.PIP_ERR_NULL
    assert lib.pip_validate(a8, 4, a8, a8, 1, -4, None, None, 0, a8, None) == _lib.PIP_ERR_SIZE


def test_tuning_validation(lib):
    from paper_2306_04316_gb300 import _lib
    t = [ctypes.c_int32() for _ in range(3)]
    assert lib.pip_get_tuning(*[ctypes.byref(x) for x in t]) == 0
    before = [x.value for x in t]
    assert lib.pip_set_tuning(100, 0, 0) == _lib.PIP_ERR_INVALID      # below 256
    assert lib.pip_set_tuning(2050, 0, 0) == _lib.PIP_ERR_INVALID     # not a multiple of 32
    assert lib.pip_set_tuning(0, 3, 0) == _lib.PIP_ERR_INVALID
    assert lib.pip_set_tuning(0, 0, 9) == _lib.PIP_ERR_INVALID
    assert lib.pip_set_tuning(1024, 4, 2) == 0
    assert lib.pip_set_small_tuning(3, 0, -1) == _lib.PIP_ERR_INVALID    # no such kernel
    assert lib.pip_set_small_tuning(-1, 64, -1) == _lib.PIP_ERR_INVALID  # slice 128 or 256
    assert lib.pip_set_small_tuning(-1, 0, 17) == _lib.PIP_ERR_INVALID
    assert lib.pip_get_tuning(*[ctypes.byref(x) for x in t]) == 0
    assert [x.value for x in t] == [1024, 4, 2]
    assert lib.pip_set_tuning(*before) == 0


def test_autotuner_grids_are_valid_tunings(lib):
    """Every shape the autotuners (and the bench's per-workload and join-step searches) may apply
    is one the library accepts, so a search never stops on PIP_ERR_INVALID."""
    from paper_2306_04316_gb300 import tuning
    s = [ctypes.c_int32() for _ in range(3)]
    t = [ctypes.c_int32() for _ in range(3)]
    assert lib.pip_get_small_tuning(*[ctypes.byref(x) for x in s]) == 0
    assert lib.pip_get_tuning(*[ctypes.byref(x) for x in t]) == 0
    try:
        for shape in tuning.DEFAULT_GRID + [(256, 4, 3), (512, 4, 3), (512, 2, 2), (1024, 4, 3), (2048, 4, 3),
                                            (4096, 4, 2)]:
            assert lib.pip_set_tuning(*shape) == 0, shape
        for shape in tuning.SMALL_GRID:
            assert lib.pip_set_small_tuning(*shape) == 0, shape
    finally:
        assert lib.pip_set_tuning(*[x.value for x in t]) == 0
        assert lib.pip_set_small_tuning(*[x.value for x in s]) == 0


def test_bin_workspace_size_grows(lib):
    """The binning workspace holds the polygons' boxes, cell table and lists (at least a 16-byte
    box, two 8-byte slots and a list entry per polygon) and the recorded (polygon, point) pairs
    (8 bytes for a quarter of the points)."""
    a = lib.pip_bin_workspace_bytes(1000, 10)
    b = lib.pip_bin_workspace_bytes(10_000_000, 100_000)
    c = lib.pip_bin_workspace_bytes(0, 100_000)
    assert 0 < a < b and 0 < c < b
    assert c >= 100_000 * (16 + 2 * 8 + 4)
    assert b - c >= 10_000_000 // 2 * 8
    # one-step workspace = index + one probe workspace
    assert b == lib.pip_bin_index_bytes(100_000) + lib.pip_bin_probe_bytes(10_000_000, 100_000)
    assert lib.pip_bin_index_bytes(-1) == 0 and lib.pip_bin_probe_bytes(-1, 10) == 0


def test_argument_checks_of_the_binning_index(lib):
    from paper_2306_04316_gb300 import _lib
    P = ctypes.c_void_p
    a8, a16 = P(0x1000), P(0x10000)
    ib, pb = lib.pip_bin_index_bytes(10), lib.pip_bin_probe_bytes(100, 10)
    assert lib.pip_bin_index(a8, a8, -1, 0, a16, ib, None) == _lib.PIP_ERR_SIZE
    assert lib.pip_bin_index(a8, a8, 10, -1, a16, ib, None) == _lib.PIP_ERR_SIZE
    assert lib.pip_bin_index(None, a8, 10, 0, a16, ib, None) == _lib.PIP_ERR_NULL
    assert lib.pip_bin_index(a8, a8, 10, 0, None, ib, None) == _lib.PIP_ERR_NULL
    assert lib.pip_bin_index(a8, a8, 10, 0, P(0x10008), ib, None) == _lib.PIP_ERR_ALIGN
    assert lib.pip_bin_index(a8, a8, 10, 0, a16, ib - 1, None) == _lib.PIP_ERR_WORKSPACE
    assert lib.pip_bin_probe_count(a8, -1, a16, ib, 10, a16, pb, a8, a8, None) == _lib.PIP_ERR_SIZE
    assert lib.pip_bin_probe_count(a8, 100, None, ib, 10, a16, pb, a8, a8, None) == _lib.PIP_ERR_NULL
    assert lib.pip_bin_probe_count(a8, 100, a16, ib, 10, a16, pb, a8, None, None) == _lib.PIP_ERR_NULL
    assert lib.pip_bin_probe_count(a8, 100, a16, ib, 10, P(0x10004), pb, a8, a8, None) == _lib.PIP_ERR_ALIGN
    assert lib.pip_bin_probe_count(a8, 100, a16, ib - 1, 10, a16, pb, a8, a8, None) == _lib.PIP_ERR_WORKSPACE
    assert lib.pip_bin_probe_count(a8, 100, a16, ib, 10, a16, pb - 1, a8, a8, None) == _lib.PIP_ERR_WORKSPACE
    assert lib.pip_bin_probe_fill(a8, 100, a16, ib, 10, a16, pb, a8, a8, -1, None, None) == _lib.PIP_ERR_SIZE
    assert lib.pip_bin_probe_fill(a8, 100, a16, ib, 10, a16, pb, a8, None, 5, None, None) == _lib.PIP_ERR_NULL
    assert lib.pip_bin_probe_fill(a8, 100, a16, ib, 10, a16, pb - 1, a8, a8, 5, None, None) == _lib.PIP_ERR_WORKSPACE


def test_argument_checks_of_the_other_entry_points(lib):
    from paper_2306_04316_gb300 import _lib
    P = ctypes.c_void_p
    a8 = P(0x1000)
    a256 = P(0x10000)
    # the printed-algorithm rules: only 1 and 2
    for alg in (0, 3, -1):
        assert lib.pip_classify_paper(a8, 4, a8, a8, 1, None, None, alg, a8, None) == _lib.PIP_ERR_INVALID
    assert lib.pip_classify_paper(a8, -1, a8, a8, 1, None, None, 1, a8, None) == _lib.PIP_ERR_SIZE
    # slab index: edges per slab 1..256, 256-byte aligned buffer, a buffer at least its fixed part
    assert lib.pip_slab_index_bytes(10, 1000, 0, 0) == 0
    assert lib.pip_slab_index_bytes(10, 1000, 257, 0) == 0
    assert lib.pip_slab_index_bytes(-1, 1000, 8, 0) == 0
    fixed = lib.pip_slab_index_bytes(10, 1000, 8, 0)
    assert 0 < fixed < lib.pip_slab_index_bytes(10, 1000, 8, 5000)
    assert lib.pip_slab_build(a8, a8, 10, 1000, 0, a256, fixed, None, None) == _lib.PIP_ERR_INVALID
    assert lib.pip_slab_build(a8, a8, 10, 1000, 8, P(0x10010), fixed, None, None) == _lib.PIP_ERR_ALIGN
    assert lib.pip_slab_build(a8, a8, 10, 1000, 8, a256, fixed - 1, None, None) == _lib.PIP_ERR_WORKSPACE
    assert lib.pip_slab_build(a8, a8, 10, -1, 8, a256, fixed, None, None) == _lib.PIP_ERR_SIZE
    assert lib.pip_slab_build(None, a8, 10, 1000, 8, a256, fixed, None, None) == _lib.PIP_ERR_NULL
    assert lib.pip_classify_slab(a8, 4, a8, a8, 1, None, None, P(0x10010), a8, None) == _lib.PIP_ERR_ALIGN
    # quantisation: positive scale, aligned arrays
    assert lib.pip_quantize_lonlat(a8, 4, 0.0, a8, None, None) == _lib.PIP_ERR_INVALID
    assert lib.pip_quantize_lonlat(a8, 4, float("nan"), a8, None, None) == _lib.PIP_ERR_INVALID
    assert lib.pip_quantize_lonlat(a8, -1, 1e7, a8, None, None) == _lib.PIP_ERR_SIZE
    assert lib.pip_quantize_lonlat(P(0x1004), 4, 1e7, a8, None, None) == _lib.PIP_ERR_ALIGN
    assert lib.pip_quantize_lonlat(None, 4, 1e7, a8, None, None) == _lib.PIP_ERR_NULL
    assert lib.pip_quantize_lonlat(None, 0, 1e7, None, None, None) == _lib.PIP_OK
    # verification mode: 0 or 1
    assert lib.pip_set_verify(2) == _lib.PIP_ERR_INVALID
    assert lib.pip_set_verify(0) == _lib.PIP_OK
