"""pip_classify_noalloc: the entry point for callers that cannot allocate device memory.

Some callers cannot let a library call cudaMalloc (their own allocator or a fixed memory
budget, paths that cannot take its synchronisation).  pip_classify_noalloc keeps
its scratch -- the list of large polygons -- in a fixed array inside the library instead.
This file is collected last so that a failure here leaves every other test already run.
The test calls the entry point through the C ABI on two calls in a row (the array keeps the
previous call's contents) and compares each output bit for bit with the CPU oracle and with
pip_classify's on the same data, in CSR and dense mode.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2306_04316_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _mixed_workload():
    """Small footprints (first kernel) and large fractal polygons (second kernel, through the
    list in the fixed array), interleaved in one CSR."""
    parts = []
    for i in range(4):
        parts.append(W.footprints(seed=300 + i, n_polys=400 + 37 * i, pts_per_poly=5 + i))
        parts.append(W.fractal(seed=400 + i, n_polys=2, m_lo=1500 + 200 * i, m_hi=1600 + 200 * i,
                               n_points=3000 + 97 * i, cell=150_000, grid=2))
    pts, po, vs, co, ids = [], [0], [], [0], []
    npts = nv = nc = 0
    for w in parts:
        pts.append(w.points)
        vs.append(w.verts)
        po += list(w.poly_offsets[1:].astype(np.int64) + nv)
        co += list(w.cand_offsets[1:].astype(np.int64) + nc)
        ids.append(w.cand_ids.astype(np.int64) + npts)
        npts += w.n_points
        nv += w.verts.shape[0]
        nc += w.n_bits
    return W.Workload("mixed", np.concatenate(pts), np.array(po, dtype=np.int32), np.concatenate(vs),
                      np.array(co, dtype=np.int32), np.concatenate(ids).astype(np.int32))


def test_noalloc_matches_pip_classify_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_04316_gb300 import _lib, api, build
    build.build_library()
    oracle.build()
    lib = _lib.load()
    w = _mixed_workload()
    assert w.n_polys <= _lib.PIP_NOALLOC_MAX_POLYS
    d = api.to_device(w)
    ref = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], d["cand_offsets"], d["cand_ids"],
                           n_cands=w.n_bits)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy().view(np.uint32)[:w.n_words]
    want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
    assert np.array_equal(ref, want)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((w.n_words,), -1, dtype=torch.int32, device="cuda")
        rc = lib.pip_classify_noalloc(d["points"].data_ptr(), w.n_points, d["poly_offsets"].data_ptr(),
                                      d["verts"].data_ptr(), w.n_polys, d["cand_offsets"].data_ptr(),
                                      d["cand_ids"].data_ptr(), out.data_ptr(), stream)
        assert rc == _lib.PIP_OK, lib.pip_status_str(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), f"call {call}: {np.count_nonzero(got != want)} words differ from the oracle"
        assert np.array_equal(got, ref), f"call {call}: {np.count_nonzero(got != ref)} words differ"
    # dense mode through the same array
    s = W.star(seed=77, m=1500, n_uniform=3000, n_special=100)
    ds = api.to_device(s)
    ref = api.pip_classify(ds["points"], ds["poly_offsets"], ds["verts"])
    want = oracle.classify(s.points, s.poly_offsets, s.verts)
    for call in range(2):
        got = torch.full_like(ref, -1)
        rc = lib.pip_classify_noalloc(ds["points"].data_ptr(), s.n_points, ds["poly_offsets"].data_ptr(),
                                      ds["verts"].data_ptr(), s.n_polys, None, None, got.data_ptr(), stream)
        assert rc == _lib.PIP_OK
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy().view(np.uint32), want), f"dense call {call} differs from the oracle"
        assert torch.equal(got, ref)
    # beyond the limit: rejected before any device work
    rc = lib.pip_classify_noalloc(d["points"].data_ptr(), w.n_points, d["poly_offsets"].data_ptr(),
                                  d["verts"].data_ptr(), _lib.PIP_NOALLOC_MAX_POLYS + 1,
                                  d["cand_offsets"].data_ptr(), d["cand_ids"].data_ptr(), out.data_ptr(), stream)
    assert rc == _lib.PIP_ERR_TOO_LARGE
