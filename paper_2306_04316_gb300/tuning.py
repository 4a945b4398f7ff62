"""Autotuner for pip_classify's kernels (not part of the paper's method).

``autotune`` times ``pip_classify`` on the caller's device arrays for every tuning tuple of the
large-polygon kernel (edge tile, candidates per thread, CTAs per SM); ``autotune_small`` for
every shape of the small-polygon kernel (lockstep, compacting or thread-per-polygon kernel,
candidates per slice, CTAs per SM).  Each keeps the fastest and stores it in a JSON cache keyed by the device name and
a shape class of the workload, so that ``apply_cached`` can set both for later calls without
timing again.  The output bits do not depend on the tuning (every tuple is covered by the GPU
parity tests); only speed does.
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_GRID = [(t, p, c) for t in (256, 512, 1024, 2048, 4096) for p in (1, 2, 4) for c in (2, 3, 4)]
# small-polygon kernel: (kernel: 0 lockstep / 1 compacting / 2 thread per polygon, candidates per slice
# (kernel 2: slice / 16 per thread), CTAs per SM, 0 = all)
SMALL_GRID = [(0, 256, 0), (0, 128, 0), (0, 256, 4), (1, 256, 0), (1, 128, 0), (1, 256, 3), (2, 256, 0),
              (2, 128, 0)]


def cache_path() -> str:
    base = os.environ.get("PIP_TUNING_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2306_04316_gb300", "tuning.json")


def shape_class(n_polys: int, n_vertices: int, n_candidates: int, dense: bool) -> str:
    """Coarse class of a workload: dense/CSR, log2 buckets of polygons, mean vertices per
    polygon and mean candidates per polygon."""
    p = max(n_polys, 1)
    mv = n_vertices / p
    mc = n_candidates / p
    return "%s-p%d-m%d-c%d" % ("dense" if dense else "csr", int(math.log2(p)), int(math.log2(max(mv, 1))),
                               int(math.log2(max(mc, 1))))


def _load_cache(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store_cache(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _key(device_name: str, cls: str) -> str:
    return f"{device_name}|{cls}"


def _search(set_fn, grid, points, poly_offsets, verts, cand_offsets, cand_ids, n_cands, reps, cache_field,
            cache):
    """Time pip_classify under each tuple of ``grid`` (applied by ``set_fn``), apply the fastest,
    store it under ``cache_field`` of this device's and shape class's cache entry."""
    import torch

    from . import api

    dense = cand_offsets is None
    n_polys = int(poly_offsets.shape[0]) - 1
    if not dense and n_cands is None:
        n_cands = int(cand_offsets[-1].item()) if n_polys > 0 else 0
    n_c = n_polys * int(points.shape[0]) if dense else int(n_cands)
    out = torch.empty(max(api.out_words(int(points.shape[0]), n_polys, None if dense else n_c), 1),
                      dtype=torch.int32, device=points.device)
    stream = torch.cuda.current_stream()
    times = {}
    for t in grid:
        set_fn(*t)
        for _ in range(2):
            api.pip_classify(points, poly_offsets, verts, cand_offsets, cand_ids, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            api.pip_classify(points, poly_offsets, verts, cand_offsets, cand_ids, out=out)
        e1.record(stream)
        e1.synchronize()
        times[t] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    set_fn(*best)
    if cache:
        path = cache_path()
        c = _load_cache(path)
        cls = shape_class(n_polys, int(verts.shape[0]), n_c, dense)
        entry = c.setdefault(_key(torch.cuda.get_device_name(points.device), cls), {})
        entry[cache_field] = list(best)
        entry[cache_field + "_ms"] = times[best]
        _store_cache(path, c)
    return best, times


def autotune(points, poly_offsets, verts, cand_offsets=None, cand_ids=None, n_cands=None, grid=None, reps=5,
             cache=True):
    """Time pip_classify for every large-polygon tuple of ``grid`` and apply the fastest; returns
    ``(best_tuple, {tuple: ms})``."""
    from . import api
    return _search(api.pip_set_tuning, grid or DEFAULT_GRID, points, poly_offsets, verts, cand_offsets, cand_ids,
                   n_cands, reps, "tuning", cache)


def autotune_small(points, poly_offsets, verts, cand_offsets=None, cand_ids=None, n_cands=None, grid=None,
                   reps=5, cache=True):
    """Time pip_classify for every small-polygon kernel shape of ``grid`` and apply the fastest;
    returns ``(best_tuple, {tuple: ms})``."""
    from . import api
    return _search(api.pip_set_small_tuning, grid or SMALL_GRID, points, poly_offsets, verts, cand_offsets,
                   cand_ids, n_cands, reps, "small", cache)


def apply_cached(n_polys: int, n_vertices: int, n_candidates: int, dense: bool, device_name: str):
    """Set the cached tuning for this device and shape class; returns it, or None if absent."""
    from . import api

    c = _load_cache(cache_path())
    entry = c.get(_key(device_name, shape_class(n_polys, n_vertices, n_candidates, dense)))
    if not entry:
        return None
    if "small" in entry:
        api.pip_set_small_tuning(*[int(x) for x in entry["small"]])
    if "tuning" not in entry:
        return None
    t = tuple(int(x) for x in entry["tuning"])
    api.pip_set_tuning(*t)
    return t
