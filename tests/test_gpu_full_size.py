"""GPU parity at the full benchmark sizes, through the same calls and default launch
configuration that bench.py times.

Footprints (1M polygons, 16M candidates), stress (1M polygons, 8M candidates) and star
(test_gpu_parity.test_star_full) are compared bit for bit with the oracle, for both kernels.
The fractal batch (8e11 pair tests) and the spatial join (100k polygons x 10M points) are
checked on seeded samples that the oracle computes one by one from the generated inputs:
sampled candidates for the fractal batch; sampled polygons for the join, whose closed-box
candidate sets and bits the oracle derives by brute force over all 10M points.
"""
import numpy as np
import pytest

import oracle
from paper_2306_04316_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import api, assert_same, check_full, gpu_bits  # noqa: E402,F401


def test_footprints_full_size(api):
    check_full(api, W.footprints(), "full size")


def test_stress_full_size(api):
    check_full(api, W.stress(), "full size")


def test_fractal_full_size_sampled(api):
    w = W.fractal()
    rng = np.random.default_rng(2306043160 + 77)
    sample = np.unique(rng.integers(0, w.n_bits, 3000))
    want = oracle.classify_sample(w.points, w.poly_offsets, w.verts, sample, w.cand_offsets, w.cand_ids)
    for exact in (False, True):
        got = oracle.unpack_bits(gpu_bits(api, w, exact), w.n_bits)[sample]
        bad = np.nonzero(got != want)[0]
        assert len(bad) == 0, f"{'exact' if exact else 'filtered'}: {len(bad)} of {len(sample)} sampled bits differ"


def test_join_full_size_sampled(api):
    w = W.join()
    d = api.to_device(w)
    co, ids = api.bin_join(d["points"], d["poly_offsets"], d["verts"])
    n_c = int(co[-1].item())
    out = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], co, ids, n_cands=n_c)
    torch.cuda.synchronize()
    co, ids = co.cpu().numpy().astype(np.int64), ids.cpu().numpy()
    bits = oracle.unpack_bits(out.cpu().numpy().view(np.uint32), n_c)
    rng = np.random.default_rng(2306043160 + 78)
    polys = np.sort(rng.choice(w.n_polys, 300, replace=False))
    counts, want_ids = oracle.bbox_join(w.points, w.poly_offsets, w.verts, polys)
    # the sampled polygons alone, with the oracle's own candidate lists
    po = w.poly_offsets.astype(np.int64)
    sub_po = np.zeros(len(polys) + 1, dtype=np.int64)
    sub_po[1:] = np.cumsum(po[polys + 1] - po[polys])
    sub_v = np.concatenate([w.verts[po[k]:po[k + 1]] for k in polys])
    sub_co = np.zeros(len(polys) + 1, dtype=np.int64)
    sub_co[1:] = np.cumsum(counts)
    want_bits = oracle.unpack_bits(
        oracle.classify(w.points, sub_po, sub_v, sub_co, want_ids.astype(np.int64)), int(sub_co[-1]))
    for i, k in enumerate(polys):
        seg = slice(co[k], co[k + 1])
        order = np.argsort(ids[seg], kind="stable")
        assert np.array_equal(ids[seg][order], want_ids[sub_co[i]:sub_co[i + 1]]), f"candidates of polygon {k}"
        assert np.array_equal(bits[seg][order], want_bits[sub_co[i]:sub_co[i + 1]]), f"bits of polygon {k}"


def test_country_full_size_sampled(api):
    """The paper-shaped batch: 17,097,823 building-like points against one 100,000-vertex
    country-like polygon (dense mode), checked on 3,000 sampled points."""
    w = W.country()
    rng = np.random.default_rng(2306043160 + 79)
    sample = np.unique(rng.integers(0, w.n_points, 3000))
    want = oracle.classify_sample(w.points, w.poly_offsets, w.verts, sample)
    got = oracle.unpack_bits(gpu_bits(api, w), w.n_bits)[sample]
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, f"{len(bad)} of {len(sample)} sampled bits differ"
