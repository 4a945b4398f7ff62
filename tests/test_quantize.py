"""float64 lon/lat -> int32 fixed point (oracle.quantize; pip_quantize_lonlat on the GPU).

Pins: ties to even on exactly representable products (a power-of-two scale), the int32 limits,
NaN and infinities; and agreement with Python's own round() of the float64 product (a different
implementation of round-half-even) on random coordinates.  The GPU test compares the library
with the oracle value for value.
"""
import math

import numpy as np
import pytest

import oracle


def test_ties_to_even_exact_products():
    v = np.array([1.25, 1.75, -1.25, -1.75, 0.25, 0.75, 2.25, 0.0, -0.0])
    out, st = oracle.quantize(v, scale=2.0)
    assert out.tolist() == [2, 4, -2, -4, 0, 2, 4, 0, 0] and st == 0


def test_limits_and_invalid_values():
    out, st = oracle.quantize([2147483647.0, -2147483648.0, 2147483647.4, -2147483648.4], scale=1.0)
    assert out.tolist() == [2147483647, -2147483648, 2147483647, -2147483648] and st == 0
    out, st = oracle.quantize([2147483647.5, 1.0], scale=1.0)          # rounds (to even) past the top
    assert out.tolist() == [0, 1] and st == 2
    out, st = oracle.quantize([float("nan"), float("inf"), -float("inf"), 3.0], scale=1.0)
    assert out.tolist() == [0, 0, 0, 3] and st == 3


def test_matches_python_round_on_random_coordinates():
    rng = np.random.default_rng(2306043160 + 95)
    v = np.concatenate([rng.uniform(-180, 180, 20000), rng.uniform(-3.3, 1.2, 20000),
                        np.round(rng.uniform(-180, 180, 5000), 7)])
    out, st = oracle.quantize(v)
    assert st == 0
    want = [round(float(x) * 1e7) for x in v]      # Python's round: ties to even, exact binary value
    assert out.astype(np.int64).tolist() == want


@pytest.mark.gpu
def test_gpu_quantize_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_04316_gb300 import api, build
    build.build_library()
    rng = np.random.default_rng(2306043160 + 96)
    v = np.concatenate([rng.uniform(-180, 180, 200_000), rng.uniform(-3.3, 1.2, 200_000),
                        np.round(rng.uniform(-180, 180, 50_000), 7),
                        np.arange(-40, 40) / 2e7 + 0.25e-7,                 # near ties
                        [214.7483647, -214.7483648, 0.0, -0.0, 1e-300, -1e-300]])
    out, st = api.quantize_lonlat(torch.from_numpy(v).cuda())
    want, wst = oracle.quantize(v)
    assert int(st.item()) == wst == 0
    assert np.array_equal(out.cpu().numpy(), want)
    bad = np.array([float("nan"), float("inf"), 215.0, 1.0])
    out, st = api.quantize_lonlat(torch.from_numpy(bad).cuda())
    want, wst = oracle.quantize(bad)
    assert int(st.item()) == wst == 3
    assert np.array_equal(out.cpu().numpy(), want)
