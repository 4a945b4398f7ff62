"""Python binding of libpip over torch tensors (device memory and streams only).

Each ``pip_*`` function below has the name of the C entry point it forwards to and only
marshals arguments: tensors become device pointers, the current torch CUDA stream becomes
the ``stream`` argument.  All classification and binning work happens in libpip's kernels.
Tensors are int32 and contiguous; ``points`` and ``verts`` are [n, 2] (x, y).  Output bits
are returned in an int32 tensor holding the uint32 words of the C ABI.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

__all__ = ["pip_classify", "pip_classify_exact", "pip_classify_paper", "pip_classify_slab", "slab_index",
           "quantize_lonlat", "pip_classify_noalloc", "bin_index", "probe_workspace", "pip_bin_probe_count",
           "pip_bin_probe_fill", "pip_bin_count", "pip_bin_fill", "bin_workspace", "bin_join",
           "pip_set_tuning", "pip_get_tuning", "pip_set_small_tuning", "pip_get_small_tuning", "pip_get_stats", "pip_reset_stats", "pip_launch_count",
           "pip_set_verify", "pip_validate", "pip_xor_words", "out_words", "to_device"]


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, name, ndim=None):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous int32 CUDA tensor")
    if ndim == 2 and (t.dim() != 2 or t.shape[1] != 2):
        raise ValueError(f"{name} must have shape [n, 2]")
    return t


def out_words(n_points: int, n_polys: int, n_cands=None) -> int:
    """Words of out_bits: ceil(C / 32) in CSR mode, n_polys * ceil(n_points / 32) dense."""
    if n_cands is None:
        return n_polys * ((n_points + 31) // 32)
    return (int(n_cands) + 31) // 32


def to_device(workload, device="cuda"):
    """Copy a ``workloads.Workload`` to int32 device tensors (a dict)."""
    d = {k: torch.from_numpy(getattr(workload, k)).to(device)
         for k in ("points", "poly_offsets", "verts")}
    if workload.cand_offsets is not None:
        d["cand_offsets"] = torch.from_numpy(workload.cand_offsets).to(device)
        d["cand_ids"] = torch.from_numpy(workload.cand_ids).to(device)
    return d


def _classify(fn_name, points, poly_offsets, verts, cand_offsets, cand_ids, out, n_cands, stream, extra=()):
    lib = _lib.load()
    _need(points, "points", 2)
    _need(poly_offsets, "poly_offsets")
    _need(verts, "verts", 2)
    _need(cand_offsets, "cand_offsets")
    _need(cand_ids, "cand_ids")
    n_points = int(points.shape[0])
    n_polys = int(poly_offsets.shape[0]) - 1
    if out is None:
        if cand_offsets is not None and n_cands is None:
            n_cands = int(cand_offsets[-1].item()) if n_polys > 0 else 0
        nw = out_words(n_points, n_polys, n_cands if cand_offsets is not None else None)
        out = torch.empty(max(nw, 1), dtype=torch.int32, device=points.device)
    _need(out, "out")
    rc = getattr(lib, fn_name)(_ptr(points), n_points, _ptr(poly_offsets), _ptr(verts), n_polys,
                               _ptr(cand_offsets), _ptr(cand_ids), *extra, _ptr(out), _stream(stream))
    _lib.check(fn_name, rc)
    return out


def pip_classify(points, poly_offsets, verts, cand_offsets=None, cand_ids=None, out=None,
                 n_cands=None, stream=None):
    """FP32-filtered exact classification (``pip_classify``); returns out_bits."""
    return _classify("pip_classify", points, poly_offsets, verts, cand_offsets, cand_ids, out,
                     n_cands, stream)


def pip_classify_exact(points, poly_offsets, verts, cand_offsets=None, cand_ids=None, out=None,
                       n_cands=None, stream=None):
    """Plain exact integer classification (``pip_classify_exact``); returns out_bits."""
    return _classify("pip_classify_exact", points, poly_offsets, verts, cand_offsets, cand_ids,
                     out, n_cands, stream)


def pip_classify_paper(points, poly_offsets, verts, cand_offsets=None, cand_ids=None, algorithm=1,
                       out=None, n_cands=None, stream=None):
    """The paper's Algorithm 1 or 2 evaluated literally (``pip_classify_paper``)."""
    return _classify("pip_classify_paper", points, poly_offsets, verts, cand_offsets, cand_ids, out,
                     n_cands, stream, extra=(int(algorithm),))


def quantize_lonlat(lonlat, scale=1e7, out=None, stream=None):
    """float64 lon/lat (CUDA tensor, any shape) -> int32 fixed point (``pip_quantize_lonlat``);
    returns (out, status) with status a one-element int32 tensor (0 = every value converted)."""
    if not (lonlat.is_cuda and lonlat.dtype == torch.float64 and lonlat.is_contiguous()):
        raise ValueError("lonlat must be a contiguous float64 CUDA tensor")
    if out is None:
        out = torch.empty(lonlat.shape, dtype=torch.int32, device=lonlat.device)
    status = torch.zeros(1, dtype=torch.int32, device=lonlat.device)
    _lib.check("pip_quantize_lonlat", _lib.load().pip_quantize_lonlat(_ptr(lonlat), lonlat.numel(), float(scale),
                                                                       _ptr(out), _ptr(status), _stream(stream)))
    return out, status


def slab_index(poly_offsets, verts, edges_per_slab=8, stream=None):
    """Build the y-slab edge index of the polygons (``pip_slab_build``) in a new device buffer,
    rebuilding once with the exact size if the first estimate (2 entries per vertex) was short.
    Returns the uint8 buffer; pass it to ``pip_classify_slab``."""
    lib = _lib.load()
    _need(poly_offsets, "poly_offsets")
    _need(verts, "verts", 2)
    n_polys = int(poly_offsets.shape[0]) - 1
    n_verts = int(verts.shape[0])
    need = torch.zeros(1, dtype=torch.int64, device=verts.device)
    cap = 2 * n_verts + 1024
    for _ in range(2):
        nbytes = int(lib.pip_slab_index_bytes(n_polys, n_verts, int(edges_per_slab), cap))
        if nbytes == 0:
            raise ValueError("bad slab index arguments")
        index = torch.empty(nbytes, dtype=torch.uint8, device=verts.device)
        _lib.check("pip_slab_build", lib.pip_slab_build(_ptr(poly_offsets), _ptr(verts), n_polys, n_verts,
                                                         int(edges_per_slab), _ptr(index), nbytes, _ptr(need),
                                                         _stream(stream)))
        n = int(need.item())
        if n <= cap:
            return index
        cap = n
    return index


def pip_classify_slab(points, poly_offsets, verts, cand_offsets=None, cand_ids=None, index=None, out=None,
                      n_cands=None, stream=None):
    """``pip_classify`` with a y-slab index (``slab_index``) for the large polygons."""
    if index is not None and not (index.is_cuda and index.is_contiguous()):
        raise ValueError("index must be the contiguous CUDA buffer returned by slab_index")
    return _classify("pip_classify_slab", points, poly_offsets, verts, cand_offsets, cand_ids, out,
                     n_cands, stream, extra=(_ptr(index),))


def pip_classify_noalloc(points, poly_offsets, verts, cand_offsets=None, cand_ids=None, out=None,
                         n_cands=None, stream=None):
    """``pip_classify`` for callers that cannot allocate device memory (``out`` is still needed:
    pass it, or let this wrapper allocate it); at most PIP_NOALLOC_MAX_POLYS polygons."""
    return _classify("pip_classify_noalloc", points, poly_offsets, verts, cand_offsets, cand_ids,
                     out, n_cands, stream)


def bin_workspace(n_points: int, n_polys: int, device="cuda"):
    lib = _lib.load()
    nbytes = int(lib.pip_bin_workspace_bytes(n_points, n_polys))
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def pip_bin_count(points, poly_offsets, verts, cell_size=0, workspace=None, cand_offsets=None,
                  d_total=None, stream=None):
    """Grid binning, counting pass: returns (cand_offsets, d_total, workspace)."""
    lib = _lib.load()
    _need(points, "points", 2)
    _need(poly_offsets, "poly_offsets")
    _need(verts, "verts", 2)
    n_points = int(points.shape[0])
    n_polys = int(poly_offsets.shape[0]) - 1
    if workspace is None:
        workspace = bin_workspace(n_points, n_polys, points.device)
    if cand_offsets is None:
        cand_offsets = torch.empty(n_polys + 1, dtype=torch.int32, device=points.device)
    if d_total is None:
        d_total = torch.empty(1, dtype=torch.int64, device=points.device)
    rc = lib.pip_bin_count(_ptr(points), n_points, _ptr(poly_offsets), _ptr(verts), n_polys,
                           int(cell_size), _ptr(workspace), workspace.numel(), _ptr(cand_offsets),
                           _ptr(d_total), _stream(stream))
    _lib.check("pip_bin_count", rc)
    return cand_offsets, d_total, workspace


def pip_bin_fill(points, poly_offsets, verts, workspace, cand_offsets, cand_ids, d_overflow=None,
                 stream=None):
    """Grid binning, fill pass: writes cand_ids (capacity = its length); returns cand_ids."""
    lib = _lib.load()
    n_points = int(points.shape[0])
    n_polys = int(poly_offsets.shape[0]) - 1
    rc = lib.pip_bin_fill(_ptr(points), n_points, _ptr(poly_offsets), _ptr(verts), n_polys,
                          _ptr(workspace), workspace.numel(), _ptr(cand_offsets), _ptr(cand_ids),
                          int(cand_ids.numel()), _ptr(d_overflow), _stream(stream))
    _lib.check("pip_bin_fill", rc)
    return cand_ids


def bin_index(poly_offsets, verts, cell_size=0, index=None, stream=None):
    """Polygon index of the binning (build once, probe with any number of point batches)."""
    lib = _lib.load()
    _need(poly_offsets, "poly_offsets")
    _need(verts, "verts", 2)
    n_polys = int(poly_offsets.shape[0]) - 1
    if index is None:
        index = torch.empty(int(lib.pip_bin_index_bytes(n_polys)), dtype=torch.uint8, device=verts.device)
    rc = lib.pip_bin_index(_ptr(poly_offsets), _ptr(verts), n_polys, int(cell_size), _ptr(index), index.numel(),
                           _stream(stream))
    _lib.check("pip_bin_index", rc)
    return index


def probe_workspace(n_points: int, n_polys: int, device="cuda"):
    lib = _lib.load()
    return torch.empty(int(lib.pip_bin_probe_bytes(n_points, n_polys)), dtype=torch.uint8, device=device)


def pip_bin_probe_count(points, index, n_polys, probe=None, cand_offsets=None, d_total=None, stream=None):
    """Count pass of one batch against a polygon index: returns (cand_offsets, d_total, probe)."""
    lib = _lib.load()
    _need(points, "points", 2)
    n_points = int(points.shape[0])
    if probe is None:
        probe = probe_workspace(n_points, n_polys, points.device)
    if cand_offsets is None:
        cand_offsets = torch.empty(n_polys + 1, dtype=torch.int32, device=points.device)
    if d_total is None:
        d_total = torch.empty(1, dtype=torch.int64, device=points.device)
    rc = lib.pip_bin_probe_count(_ptr(points), n_points, _ptr(index), index.numel(), int(n_polys), _ptr(probe),
                                 probe.numel(), _ptr(cand_offsets), _ptr(d_total), _stream(stream))
    _lib.check("pip_bin_probe_count", rc)
    return cand_offsets, d_total, probe


def pip_bin_probe_fill(points, index, n_polys, probe, cand_offsets, cand_ids, d_overflow=None, stream=None):
    """Fill pass of one batch (after its count pass on the same probe workspace)."""
    lib = _lib.load()
    n_points = int(points.shape[0])
    rc = lib.pip_bin_probe_fill(_ptr(points), n_points, _ptr(index), index.numel(), int(n_polys), _ptr(probe),
                                probe.numel(), _ptr(cand_offsets), _ptr(cand_ids), int(cand_ids.numel()),
                                _ptr(d_overflow), _stream(stream))
    _lib.check("pip_bin_probe_fill", rc)
    return cand_ids


def bin_join(points, poly_offsets, verts, cell_size=0, stream=None):
    """Both binning passes with one host read of the candidate total in between."""
    co, tot, ws = pip_bin_count(points, poly_offsets, verts, cell_size, stream=stream)
    total = int(tot.item())
    ids = torch.empty(max(total, 1), dtype=torch.int32, device=points.device)
    pip_bin_fill(points, poly_offsets, verts, ws, co, ids[:total] if total else ids[:0], stream=stream)
    return co, ids[:total]


def pip_set_tuning(edge_tile=0, pts_per_thread=0, ctas_per_sm=0):
    _lib.check("pip_set_tuning", _lib.load().pip_set_tuning(edge_tile, pts_per_thread, ctas_per_sm))


def pip_get_tuning():
    v = [ctypes.c_int32() for _ in range(3)]
    _lib.check("pip_get_tuning", _lib.load().pip_get_tuning(*[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def pip_set_small_tuning(kernel=-1, slice=0, ctas_per_sm=-1):
    """Small-polygon kernel: 0 = lockstep rounds, 1 = compacting, 2 = thread per polygon;
    candidates per slice (128, 256; kernel 2 takes slice / 16 per thread); resident CTAs per SM
    (0 = as many as fit).  -1 / 0 keep a value."""
    _lib.check("pip_set_small_tuning", _lib.load().pip_set_small_tuning(kernel, slice, ctas_per_sm))


def pip_get_small_tuning():
    v = [ctypes.c_int32() for _ in range(3)]
    _lib.check("pip_get_small_tuning", _lib.load().pip_get_small_tuning(*[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def pip_xor_words(dst, src, stream=None):
    """dst ^= src on the device (int32 tensors of the same length; ``pip_xor_words``)."""
    for t, n in ((dst, "dst"), (src, "src")):
        if not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous():
            raise ValueError(f"{n} must be a contiguous int32 CUDA tensor")
    if dst.numel() != src.numel():
        raise ValueError("dst and src must have the same length")
    _lib.check("pip_xor_words", _lib.load().pip_xor_words(_ptr(dst), _ptr(src), dst.numel(), _stream(stream)))
    return dst


def pip_get_stats() -> dict:
    s = _lib.PipStats()
    _lib.check("pip_get_stats", _lib.load().pip_get_stats(ctypes.byref(s)))
    return {f: int(getattr(s, f)) for f, _ in _lib.PipStats._fields_}


def pip_set_verify(on: bool):
    """Verification mode: every trusted fast-path decision is rechecked exactly and
    disagreements are counted in pip_get_stats()["filter_errors"]."""
    _lib.check("pip_set_verify", _lib.load().pip_set_verify(1 if on else 0))


def pip_launch_count() -> int:
    """Kernels the library has enqueued since it was loaded (graph replays not counted)."""
    return int(_lib.load().pip_launch_count())


def pip_reset_stats():
    _lib.check("pip_reset_stats", _lib.load().pip_reset_stats())


def pip_validate(points, poly_offsets, verts, cand_offsets=None, cand_ids=None, stream=None) -> int:
    """Device-side data check; returns the status mask (0 = valid).  Synchronises."""
    lib = _lib.load()
    st = torch.zeros(1, dtype=torch.int32, device=points.device)
    n_ids = int(cand_ids.numel()) if cand_ids is not None else 0
    rc = lib.pip_validate(_ptr(points), int(points.shape[0]), _ptr(poly_offsets), _ptr(verts),
                          int(poly_offsets.shape[0]) - 1, int(verts.shape[0]), _ptr(cand_offsets),
                          _ptr(cand_ids), n_ids, _ptr(st), _stream(stream))
    _lib.check("pip_validate", rc)
    return int(st.item())
