#!/usr/bin/env python
"""Benchmark: point-edge tests/s and points classified/s of pip_classify on one GB300.

Workload (N = 1): the 1M building-footprint batch -- 1,000,000 polygons (log-normal 4-64
vertices, mean ~7), 16 candidate points per polygon (16M candidates), int32 1e-7-degree
coordinates in Ghana's lon/lat box; synthetic and seeded.  One step = one pip_classify call
over the whole batch (all steps of the method: candidate fetch, edge staging and local
frame, straddle test, FP32 side test with exact fallback, parity, ballot pack).  Under
torchrun each rank classifies its own batch (seed + rank): weak scaling, no collective on
the data path.  The inputs (~258 MB) exceed the 129 MB L2, so no flush is needed between
steps.

Printed JSON line: value = pair tests/s over the whole job (device-timed, inputs resident);
e2e = the same metric through the public API with host buffers (H2D of every input and D2H
of the bits inside the timed region); roofline of the classify kernel against measured HBM
bandwidth; the CPU oracle as the baseline; SM clocks sampled during the timed region.

``--impl reference`` times the CPU oracle (the reference implementation of the method in
this repository) on a bounded sample of the same workload and prints the same line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "point-edge tests/s and points classified/s (1 GB300), % of roofline, 0 mismatches"
UNIT = "pair-tests/s"


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def dist_setup(world, backend="nccl"):
    """torch.distributed for N > 1 (one process per GPU, launched by torchrun), else None."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend)
    return dist


def max_over_ranks(dist, value, device="cuda"):
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, device="cuda"):
    """The total of a per-rank count over all ranks (each rank's batch has its own data)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_all_ranks, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_all_ranks / (ms / 1000.0)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        time.sleep(0.25)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_baseline(w, target_s=10.0, max_reps=20, max_pairs=2e10):
    """The CPU oracle on the whole batch, repeated until ~target_s of CPU work; for batches
    above max_pairs pair tests, on a seeded sample of candidates instead."""
    import numpy as np
    import oracle
    threads = oracle.default_threads()
    oracle.build()
    T = w.pair_tests()
    if T <= max_pairs:
        reps, t_total = 0, 0.0
        while reps < max_reps and (t_total < target_s or reps == 0):
            t0 = time.perf_counter()
            oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids, threads=threads)
            t_total += time.perf_counter() - t0
            reps += 1
        return {"value": T * reps / t_total, "unit": UNIT, "cores": threads, "kind": "oracle",
                "sample": f"whole {w.name} batch ({w.n_polys} polygons, {w.n_candidates} candidates, "
                          f"{T} pair tests) x {reps} runs, {t_total:.1f} s",
                "points_per_s": w.n_candidates * reps / t_total}
    # sampled: candidates drawn uniformly, classified one by one (threaded over the sample);
    # a short probe sizes the sample to about target_s of CPU work
    rng = np.random.default_rng(12345)
    m = np.diff(w.poly_offsets.astype(np.int64))
    owner = None if w.dense else np.repeat(np.arange(w.n_polys), np.diff(w.cand_offsets.astype(np.int64)))

    def draw(n):
        if w.dense:
            W32 = 32 * ((w.n_points + 31) // 32)
            s_ = np.unique(rng.integers(0, w.n_polys, n) * W32 + rng.integers(0, w.n_points, n))
            return s_, int(m[s_ // W32].sum())
        s_ = np.sort(rng.choice(len(owner), size=min(n, len(owner)), replace=False))
        return s_, int(m[owner[s_]].sum())

    probe, probe_pairs = draw(max(64, int(w.n_candidates * 1e8 / T)))
    t0 = time.perf_counter()
    _threaded_sample(w, probe, threads)
    rate = probe_pairs / max(1e-9, time.perf_counter() - t0)
    sample, pairs = draw(max(64, int(len(probe) * rate * target_s / max(1, probe_pairs))))
    t0 = time.perf_counter()
    _threaded_sample(w, sample, threads)
    dt = time.perf_counter() - t0
    return {"value": pairs / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(sample)} seeded candidates of the {w.name} batch ({pairs} pair tests), {dt:.1f} s",
            "points_per_s": len(sample) / dt}


def _threaded_sample(w, sample, threads):
    import numpy as np
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    parts = np.array_split(sample, threads)
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda s_: oracle.classify_sample(w.points, w.poly_offsets, w.verts, s_, w.cand_offsets,
                                                      w.cand_ids), parts))


KERNEL_SOURCES = ["paper_2306_04316_gb300/csrc/pip_filtered.cu", "paper_2306_04316_gb300/csrc/pip_small.cu",
                  "paper_2306_04316_gb300/csrc/pip_tpp.cu",
                  "paper_2306_04316_gb300/csrc/pip_edge.cuh", "paper_2306_04316_gb300/csrc/pip_device.cuh",
                  "paper_2306_04316_gb300/csrc/pip_launch.h"]


SMALL_KERNEL_NAMES = {0: "k_pip_warp", 1: "k_pip_cmp", 2: "k_pip_tpp"}   # pip_set_small_tuning's kernels


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, kernel="k_pip_warp"):
    """DRAM bytes per launch of the classify kernel from the committed ncu summary, or None when
    the kernel sources changed since that capture (or no summary covers this workload)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("- ") and ": " in line:
                k, v = line[2:].split(": ", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel source sha256[:16]") != kernel_source_hash():
        return None
    try:
        return int(vals["dram bytes per launch (read + write)"])
    except (KeyError, ValueError):
        return None


def make_workload(name, rank, scale):
    from paper_2306_04316_gb300 import workloads as W
    if name == "footprints":
        return W.footprints(seed=W.BASE_SEED + 2 + 1000 * rank, n_polys=int(1_000_000 * scale))
    if name == "stress":
        return W.stress(seed=W.BASE_SEED + 5 + 1000 * rank, n_polys=int(1_000_000 * scale))
    if name == "star":
        return W.star(seed=W.BASE_SEED + 1 + 1000 * rank)
    if name == "fractal":
        return W.fractal(seed=W.BASE_SEED + 4 + 1000 * rank, n_points=int(10_000_000 * scale))
    if name == "country":
        return W.country(seed=W.BASE_SEED + 6 + 1000 * rank, n_points=max(1, int(W.PAPER_N_POINTS * scale)))
    raise SystemExit(f"unknown workload {name}")


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w = make_workload(args.workload, 0, 1.0)
    # a bounded sample: the leading polygons (or points, in dense mode) of the batch, sized from
    # a short probe so that warm-up plus timed steps take about two minutes of CPU work in total
    threads = oracle.default_threads()
    probe = w.bounded(2e8)
    t0 = time.perf_counter()
    oracle.classify(probe.points, probe.poly_offsets, probe.verts, probe.cand_offsets, probe.cand_ids, threads=threads)
    rate = probe.pair_tests() / max(1e-9, time.perf_counter() - t0)
    sub = w.bounded(rate * 120.0 / max(1, args.steps + args.warmup))
    steps_t = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.classify(sub.points, sub.poly_offsets, sub.verts, sub.cand_offsets, sub.cand_ids, threads=threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            steps_t.append(dt)
    T = sub.pair_tests()
    tot = sum(steps_t)
    value = T * len(steps_t) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(steps_t),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": f"{w.name}: {w.n_polys} polygons, {w.n_candidates} candidates",
                                             "pair_tests_per_step": T, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"leading part of the {w.name} batch per step: {sub.n_polys} of {w.n_polys} "
                                       f"polygons, {sub.n_candidates} candidates, {T} pair tests"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "points_per_s": sub.n_candidates * len(steps_t) / tot}
    print(json.dumps(line), flush=True)
    return 0


def arithmetic_of(w):
    """The arithmetic the filtered kernels use on this workload, from the polygons' boxes: exact
    int32 for boxes below 2^30 with width x height below 2^30, exact int64 for boxes below 2^31,
    FP32 (with an exact integer recheck) above and for polygons of more than 256 vertices;
    "i32+i64" when both integer kinds occur, and so on."""
    import numpy as np
    po = w.poly_offsets.astype(np.int64)
    m = np.diff(po)
    keep = m > 0
    if not keep.any():
        return "i32"
    v = w.verts.astype(np.int64)
    starts = po[:-1][keep]
    W_ = np.maximum.reduceat(v[:, 0], starts) - np.minimum.reduceat(v[:, 0], starts)
    H_ = np.maximum.reduceat(v[:, 1], starts) - np.minimum.reduceat(v[:, 1], starts)
    i32 = (W_ < 2**30) & (H_ < 2**30) & (W_ * H_ < 2**30)
    i64 = ~i32 & (W_ < 2**31) & (H_ < 2**31)
    large = (m[keep] > 256)
    kinds = []
    if (i32 & ~large).any():
        kinds.append("i32")
    if (i64 & ~large).any():
        kinds.append("i64")
    if ((~i32 & ~i64) | large).any():   # large polygons always take the FP32 filter
        kinds.append("f32")
    return "+".join(kinds)


def run_join(args, rank, world, quiet=False):
    """Spatial join: 100k footprint polygons against 20 batches of 10M clustered points; one
    step = one replay of a CUDA graph that bins and classifies all 20 batches.  With ``quiet``
    (a compact measurement for another workload's line) the line is returned, not printed, and
    the end-to-end leg, the CPU baseline and the clock sampler are skipped."""
    import numpy as np
    import torch
    from paper_2306_04316_gb300 import api, build as pbuild, workloads as W

    pbuild.build_library()
    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    dist = None if quiet else dist_setup(world)
    nb = args.batches
    n_pts = int(10_000_000 * args.scale)
    seed = W.BASE_SEED + 3 + 1000 * rank
    clusters, po, v = W.join_polygons(seed=seed, n_polys=int(100_000 * max(args.scale, 0.01)))
    P = len(po) - 1
    d_po, d_v = torch.from_numpy(po).cuda(), torch.from_numpy(v).cuda()
    host_pts = [W.join_points(clusters, seed + 1000 + b, n_pts) for b in range(nb)]
    d_pts = [torch.from_numpy(x).cuda() for x in host_pts]
    stream = torch.cuda.Stream()
    # a step builds the polygon index once; the batches then probe it on several streams (each
    # with its own probe workspace) so that their latency-bound kernels overlap; the graph forks
    # from and joins back to `stream`
    ns = max(1, min(args.streams, nb))
    streams = [torch.cuda.Stream() for _ in range(ns)]
    index = api.bin_index(d_po, d_v, stream=stream)
    probes = [api.probe_workspace(n_pts, P) for _ in range(ns)]
    co = [torch.empty(P + 1, dtype=torch.int32, device="cuda") for _ in range(nb)]
    tot = [torch.empty(1, dtype=torch.int64, device="cuda") for _ in range(nb)]
    with torch.cuda.stream(stream):
        totals = []
        for b in range(nb):
            api.pip_bin_probe_count(d_pts[b], index, P, probe=probes[0], cand_offsets=co[b], d_total=tot[b],
                                    stream=stream)
            stream.synchronize()
            totals.append(int(tot[b].item()))
    cap = int(max(totals) * 1.1) + 1024
    ids = [torch.empty(cap, dtype=torch.int32, device="cuda") for _ in range(nb)]
    outs = [torch.empty(cap // 32 + 1, dtype=torch.int32, device="cuda") for _ in range(nb)]
    ovf = torch.zeros(nb, dtype=torch.int32, device="cuda")

    # pinned host buffers of the end-to-end step: the batches' points in, their bits and candidate
    # CSR out
    with_e2e = not args.no_e2e and not quiet
    if with_e2e:
        h_pts = [torch.from_numpy(x).pin_memory() for x in host_pts]
        h_out = [torch.empty(o.numel(), dtype=torch.int32).pin_memory() for o in outs]
        h_ids = [torch.empty(t_, dtype=torch.int32).pin_memory() for t_ in totals]
        h_co = [torch.empty(P + 1, dtype=torch.int32).pin_memory() for _ in range(nb)]

    def one_pass(classify=True, io=False):
        api.bin_index(d_po, d_v, index=index, stream=stream)
        for s_ in streams:
            s_.wait_stream(stream)
        for b in range(nb):
            s_, q_ = streams[b % ns], probes[b % ns]
            if io:   # this batch's points from the host, on the batch's stream
                with torch.cuda.stream(s_):
                    d_pts[b].copy_(h_pts[b], non_blocking=True)
            api.pip_bin_probe_count(d_pts[b], index, P, probe=q_, cand_offsets=co[b], d_total=tot[b], stream=s_)
            api.pip_bin_probe_fill(d_pts[b], index, P, q_, co[b], ids[b], d_overflow=ovf[b:b + 1], stream=s_)
            if classify:
                api.pip_classify(d_pts[b], d_po, d_v, co[b], ids[b], out=outs[b], stream=s_)
            if io:   # its bits and candidate lists back, while the other streams compute
                with torch.cuda.stream(s_):
                    h_co[b].copy_(co[b], non_blocking=True)
                    h_ids[b].copy_(ids[b][:totals[b]], non_blocking=True)
                    h_out[b].copy_(outs[b], non_blocking=True)
        for s_ in streams:
            stream.wait_stream(s_)

    with torch.cuda.stream(stream):
        one_pass()
        one_pass()
    stream.synchronize()
    assert int(ovf.sum().item()) == 0
    # the small- and large-polygon kernels' shapes, picked by the autotuner on the first batch
    from paper_2306_04316_gb300 import tuning
    best_s, times_s = tuning.autotune_small(d_pts[0], d_po, d_v, co[0], ids[0], n_cands=totals[0], cache=False)
    best, times = tuning.autotune(d_pts[0], d_po, d_v, co[0], ids[0], n_cands=totals[0], cache=False)
    autotuned = {"best": list(best), "candidates": len(times), "best_ms": times[best],
                 "small": {"best": list(best_s), "candidates": len(times_s), "best_ms": times_s[best_s]}}
    # The large-polygon kernel's tuning also sets how much of each SM its CTAs hold while they wait
    # for the small-polygon kernel before them (programmatic dependent launch); with four streams
    # overlapping, that matters more than the single-call times above, which are all within noise
    # here.  So a few tunings (the single-call pick and one per edge tile) are timed on the step.
    step_ms = {}
    for t in [tuple(best)] + [t for t in ((256, 4, 3), (512, 2, 2), (1024, 4, 3), (2048, 4, 3)) if t != tuple(best)]:
        api.pip_set_tuning(*t)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            one_pass(True)
        with torch.cuda.stream(stream):
            g.replay()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                g.replay()
            e1.record(stream)
            stream.synchronize()
        step_ms[t] = e0.elapsed_time(e1) / 3
        del g
    best_step = min(step_ms, key=step_ms.get)
    api.pip_set_tuning(*best_step)
    autotuned["step"] = {"best": list(best_step), "ms": {",".join(map(str, k)): v for k, v in step_ms.items()}}
    m = np.diff(po.astype(np.int64))
    T = sum(int((m * np.diff(c.cpu().numpy().astype(np.int64))).sum()) for c in co)
    C = sum(int(c[-1].item()) for c in co)
    graphs, per_replay = {}, {}
    for name, cls in (("full", True), ("binning", False)):
        g = torch.cuda.CUDAGraph()
        l0 = api.pip_launch_count()
        with torch.cuda.graph(g, stream=stream):
            one_pass(cls)
        per_replay[name] = api.pip_launch_count() - l0
        graphs[name] = g
    g_e2e = None
    if with_e2e:
        g_e2e = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_e2e, stream=stream):
            one_pass(True, io=True)
    res = {}
    for name, g in graphs.items():
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                g.replay()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(_env_int("LOCAL_RANK", 0)) if name == "full" and not quiet else None
        if sampler:
            sampler.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                g.replay()
        e1.record(stream)
        stream.synchronize()
        if dist:
            dist.barrier()
        res[name] = (max_over_ranks(dist, e0.elapsed_time(e1)) / args.steps, sampler.stop() if sampler else None)
    ms, clocks = res["full"]
    T_all = sum_over_ranks(dist, T)
    bin_ms = res["binning"][0]
    # end to end: one replay of a graph in which every batch's stream copies its points from
    # pinned host memory, bins and classifies them, and copies its bits and candidate CSR back,
    # so that copies overlap the other batches' kernels
    e2e = None
    if g_e2e is not None:
        h2d = sum(x.numel() * x.element_size() for x in h_pts)
        d2h = sum(x.numel() * 4 for x in h_out) + sum(x.numel() * 4 for x in h_ids) + nb * 4 * (P + 1)

        def e2e_step():
            g_e2e.replay()

        n_e = max(1, min(args.e2e_steps, 5))
        with torch.cuda.stream(stream):
            e2e_step()
            stream.synchronize()
            if dist:
                dist.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n_e):
                e2e_step()
            e1.record(stream)
            stream.synchronize()
        e2e_ms = max_over_ranks(dist, e0.elapsed_time(e1)) / n_e
        e2e = {"value": job_rate(T_all, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms}
    # algorithmic bytes of a step (what any binning + classification must move, independent of
    # how it is done): the polygons' vertices read once for the index; per batch the points read
    # once and the CSR written (offsets, ids); the classification reads vertices, offsets, ids
    # and points and writes the bits
    V = int(po[-1])
    classify_bytes = 8 * V * nb + 8 * (P + 1) * nb + 12 * C + C // 8
    bin_bytes = 8 * V + nb * (8 * n_pts + 4 * (P + 1)) + 4 * C
    join_bytes = classify_bytes + bin_bytes
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not quiet:
        sub_p = min(P, 2000)
        sub = W.Workload("join-sample", host_pts[0][:1_000_000], po[:sub_p + 1], v[:int(po[sub_p])])
        co_s, ids_s = W.bbox_csr(sub.poly_offsets.astype(np.int64), sub.verts, sub.points)
        cpu = oracle_baseline(sub.with_csr(co_s, ids_s, name="join-sample"))
        cpu["sample"] = f"first {sub_p} polygons x first 1M points of batch 0 (numpy closed-bbox CSR): " + cpu["sample"]
    if rank == 0:
        line = {"metric": METRIC, "value": job_rate(T_all, ms), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": arithmetic_of(W.Workload("join", host_pts[0][:1], po, v)),
                "data": "synthetic",
                "config": {"workload": f"join: {P} polygons x {nb} batches of {n_pts} clustered points, "
                                       f"{C} candidates from GPU binning, one CUDA-graph replay per step "
                                       f"({ns} streams)",
                           "pair_tests_per_step": T, "candidates_per_step": C, "binning_ms_per_step": bin_ms,
                           "classify_ms_per_step": ms - bin_ms, "tuning": list(api.pip_get_tuning()),
                           "small_tuning": list(api.pip_get_small_tuning()),
                           "autotuned": autotuned, "l2": "inputs larger than L2 (no flush)"},
                "points_per_s": job_rate(nb * n_pts * world, ms), "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": per_replay["full"] * args.steps,
                "roofline": {"bound": "hbm", "achieved": join_bytes / (ms / 1000.0) / 1e9, "peak": hbm,
                             "unit": "GB/s", "frac": join_bytes / (ms / 1000.0) / 1e9 / hbm, "traffic": None,
                             "peak_source": peak_kind, "kernel": f"binning + {SMALL_KERNEL_NAMES.get(best_s[0], 'k_pip_warp')} + k_pip_large (whole step)",
                             "algorithmic_bytes": join_bytes, "kernel_ms": ms},
                "e2e": e2e}
        if quiet:
            return line
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_strong(args, rank, world):
    """One global batch split across the ranks (strong scaling): the footprint and stress
    batches by contiguous polygon ranges balanced by pair tests, each rank writing its bits at
    their global positions of a zeroed full-size output, combined by an integer SUM all-reduce
    (the ranks' bits are disjoint); the fractal and country batches by edge pieces closed
    through each polygon's first vertex, combined by all-gather and XOR.  A step is the memset,
    the rank's pip_classify call and the combine; the time is the slowest rank's."""
    import numpy as np
    import torch
    from paper_2306_04316_gb300 import api, build as pbuild, shard

    pbuild.build_library()
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = dist_setup(world)
    w = make_workload(args.workload, 0, args.scale)   # the same global batch on every rank
    T, C = w.pair_tests(), w.n_candidates
    by_edges = w.dense or args.workload in ("fractal", "country")
    pts = torch.from_numpy(w.points).cuda()
    if by_edges:
        ppo, pv = shard.edge_pieces(w.poly_offsets, w.verts, world)[rank]
        po, v = torch.from_numpy(ppo).cuda(), torch.from_numpy(pv).cuda()
        co = None if w.dense else torch.from_numpy(w.cand_offsets).cuda()
        ids = None if w.dense else torch.from_numpy(w.cand_ids).cuda()
        part = f"edge pieces closed through R_0, {world} per polygon"
    else:
        b = shard.polygon_ranges(w.poly_offsets, w.cand_offsets, world)
        p0, p1 = int(b[rank]), int(b[rank + 1])
        po = torch.from_numpy(w.poly_offsets[p0:p1 + 1]).cuda()
        v = torch.from_numpy(w.verts).cuda()
        co = torch.from_numpy(w.cand_offsets[p0:p1 + 1]).cuda()
        ids = torch.from_numpy(w.cand_ids).cuda()
        part = "contiguous polygon ranges balanced by pair tests"
    out = torch.zeros(max(w.n_words, 1), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    n_bits = None if w.dense else w.n_bits

    def step():
        out.zero_()
        if int(po.shape[0]) > 1:
            api.pip_classify(pts, po, v, co, ids, out=out, n_cands=n_bits)
        if by_edges:
            shard.combine_xor(out, dist)
        else:
            shard.combine_disjoint(out, dist)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(dist, e0.elapsed_time(e1) / args.steps)
    if rank == 0:
        line = {"metric": METRIC, "value": job_rate(T, ms), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": None, "dtype": arithmetic_of(w), "data": "synthetic",
                "config": {"workload": f"{w.name}: {w.n_polys} polygons, {C} candidates (one global batch)",
                           "partition": part, "pair_tests_per_step": T,
                           "timing": "memset + pip_classify + combine per step, direct calls"},
                "points_per_s": job_rate(C, ms), "gpu_launches": None}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def roofline_of(T, B, kern_ms, peaks, peak_kind, n_sm, kernel, traffic=None):
    """Roofline of a classify step: t_roof = max(T / P_pair, B / BW), P_pair = N_SM x 128 lanes x
    f_max / 4 lane-instructions per pair, BW = the measured HBM copy bandwidth; the bound is
    whichever term is larger, and frac = achieved / peak for that term."""
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    pair_peak = n_sm * 128 * f_max / 4.0
    hbm = float(peaks["hbm_gbs"])
    if B / (hbm * 1e9) >= T / pair_peak:
        achieved = B / (kern_ms / 1000.0) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "peak_source": peak_kind, "kernel": kernel, "algorithmic_bytes": B,
                "kernel_ms": kern_ms}
    achieved = T / (kern_ms / 1000.0)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": pair_peak / 1e12, "unit": "Tpair/s",
            "frac": achieved / pair_peak, "traffic": traffic,
            "peak_source": f"{n_sm} SMs x 128 lanes x {f_max / 1e6:.0f} MHz / 4 lane-instructions per pair",
            "kernel": kernel, "algorithmic_bytes": B, "kernel_ms": kern_ms}


def time_graph_steps(call, stream, steps, warmup, flush_bytes=0):
    """Mean CUDA-event time (ms) of one replay of a graph holding ``call``, timed on ``stream``
    after warm-up; with flush_bytes, that many bytes are written between steps, outside the
    timed intervals (an L2 flush)."""
    import statistics as st_
    import torch
    with torch.cuda.stream(stream):
        for _ in range(2):
            call()
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        call()
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda") if flush_bytes else None
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            g.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for e0, e1 in ev:
            if flush is not None:
                flush.zero_()
            e0.record(stream)
            g.replay()
            e1.record(stream)
    torch.cuda.synchronize()
    return st_.mean(e0.elapsed_time(e1) for e0, e1 in ev)


def other_configs(args, peaks, peak_kind, n_sm):
    """Compact device-timed measurements of the other workloads at their full sizes (one GPU, no
    CPU baseline): star, stress, fractal, country with pip_classify, the join with its whole
    binning + classification step."""
    import gc
    import torch
    from paper_2306_04316_gb300 import api
    from paper_2306_04316_gb300 import tuning
    res = {}
    stream = torch.cuda.Stream()
    small0, large0 = api.pip_get_small_tuning(), api.pip_get_tuning()
    large_grid = [(256, 4, 3), (512, 4, 3), (2048, 4, 3), (4096, 4, 2)]
    for name, steps in (("star", 20), ("stress", 20), ("fractal", 4), ("country", 3)):
        w = make_workload(name, 0, 1.0)
        T, B = w.pair_tests(), w.algorithmic_bytes()
        d = api.to_device(w)
        out = torch.empty(w.n_words, dtype=torch.int32, device="cuda")
        co, ci = d.get("cand_offsets"), d.get("cand_ids")
        # each workload's kernel shapes picked on its own batch: the small-polygon kernel always,
        # the large-polygon kernel's tuning where its polygons carry the work
        n_c = None if w.dense else w.n_bits
        api.pip_set_small_tuning(*small0)
        api.pip_set_tuning(*large0)
        tuned = {"small": list(tuning.autotune_small(d["points"], d["poly_offsets"], d["verts"], co, ci,
                                                     n_cands=n_c, reps=3, cache=False)[0])}
        if name in ("star", "fractal", "country"):
            tuned["large"] = list(tuning.autotune(d["points"], d["poly_offsets"], d["verts"], co, ci, n_cands=n_c,
                                                  grid=large_grid, reps=2, cache=False)[0])

        def call():
            api.pip_classify(d["points"], d["poly_offsets"], d["verts"], co, ci, out=out)
        api.pip_reset_stats()
        ms = time_graph_steps(call, stream, steps, 3, 256 * 2**20 if B < 160 * 10**6 else 0)
        stt = api.pip_get_stats()
        roof = roofline_of(T, B, ms, peaks, peak_kind, n_sm, "pip_classify")
        res[name] = {"workload": f"{w.name}: {w.n_polys} polygons, {w.n_candidates} candidates, "
                                 f"{w.verts.shape[0]} vertices", "steps": steps, "ms_per_step": ms,
                     "pair_tests_per_s": T / (ms / 1000.0), "points_per_s": w.n_candidates / (ms / 1000.0),
                     "roofline": {k: roof[k] for k in ("bound", "achieved", "peak", "unit", "frac")},
                     "dtype": arithmetic_of(w),
                     "fallback_fraction": stt["fallback_points"] / stt["candidates"] if stt["candidates"] else None,
                     "wait_timeouts": stt["wait_timeouts"], "autotuned": tuned}
        del d, out, w
        gc.collect()
        torch.cuda.empty_cache()
    api.pip_set_small_tuning(*small0)
    api.pip_set_tuning(*large0)
    jargs = argparse.Namespace(**vars(args))
    jargs.steps, jargs.warmup, jargs.scale = 3, 3, 1.0
    jl = run_join(jargs, 0, 1, quiet=True)
    res["join"] = {"workload": jl["config"]["workload"], "steps": 3, "ms_per_step": jl["ms_per_step"],
                   "pair_tests_per_s": jl["value"], "points_per_s": jl["points_per_s"],
                   "binning_ms_per_step": jl["config"]["binning_ms_per_step"],
                   "roofline": {k: jl["roofline"][k] for k in ("bound", "achieved", "peak", "unit", "frac")},
                   "dtype": jl["dtype"], "autotuned": jl["config"]["autotuned"]}
    api.pip_set_small_tuning(*small0)
    api.pip_set_tuning(*large0)
    gc.collect()
    torch.cuda.empty_cache()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="footprints", choices=["footprints", "stress", "star", "fractal", "join", "country"])
    ap.add_argument("--kernel", default="filtered", choices=["filtered", "exact"])
    ap.add_argument("--index", default="none", choices=["none", "slab"],
                    help="slab: classify through a y-slab edge index of the large polygons (built once, "
                         "outside the timed region); changes the number of pair tests, so the line reports "
                         "points/s instead")
    ap.add_argument("--edges-per-slab", type=int, default=8)
    ap.add_argument("--verify", action="store_true",
                    help="after timing, one pass in verification mode: every trusted fast-path decision "
                         "rechecked exactly; reports the disagreements (must be 0)")
    ap.add_argument("--semantics", default="halfopen", choices=["halfopen", "alg1", "alg2"],
                    help="alg1/alg2: time the paper's printed Algorithm 1 or 2 (pip_classify_paper) and "
                         "count the bits where it differs from the half-open rule")
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the full batch (tests only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="weak: every rank classifies its own batch; strong: one global batch split across "
                         "the ranks (polygon ranges, or edge pieces for the large polygons) and combined")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the compact measurements of the other workloads on the footprint line")
    ap.add_argument("--no-graph", action="store_true",
                    help="time direct calls instead of replays of a CUDA graph holding one call")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--batches", type=int, default=20, help="join workload: point batches per step")
    ap.add_argument("--streams", type=int, default=4,
                    help="join workload: streams the batches are spread over inside the graph")
    ap.add_argument("--tuning", default="", help="edge_tile,pts_per_thread,ctas_per_sm (0 = keep)")
    ap.add_argument("--small-tuning", default="",
                    help="small-polygon kernel: kernel,slice,ctas_per_sm (kernel 1 = compacting, 0 = lockstep; "
                         "-1 / 0 keep a value)")
    ap.add_argument("--autotune", action="store_true",
                    help="also pick the large-polygon kernel's tuning with the autotuner before timing "
                         "(always on for --workload join)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's small-polygon kernel shape instead of tuning it on the batch")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "join":
        return run_join(args, rank, world)
    if args.scaling == "strong":
        return run_strong(args, rank, world)

    import numpy as np
    import torch
    from paper_2306_04316_gb300 import api, build as pbuild

    pbuild.build_library()
    torch.cuda.set_device(local)
    if args.tuning:
        api.pip_set_tuning(*[int(x) for x in args.tuning.split(",")])
    if args.small_tuning:
        api.pip_set_small_tuning(*[int(x) for x in args.small_tuning.split(",")])
    dist = dist_setup(world)

    w = make_workload(args.workload, rank, args.scale)
    T = w.pair_tests()
    B = w.algorithmic_bytes()
    d = api.to_device(w)
    n_words = w.n_words
    out = torch.empty(n_words, dtype=torch.int32, device="cuda")
    autotuned = None
    if args.kernel == "filtered" and args.semantics == "halfopen":
        from paper_2306_04316_gb300 import tuning
        n_c = None if w.dense else w.n_bits
        autotuned = {}
        if not args.small_tuning and not args.no_autotune:
            # the small-polygon kernel's shape, picked on this batch (a few ms of timed calls)
            best, times = tuning.autotune_small(d["points"], d["poly_offsets"], d["verts"], d.get("cand_offsets"),
                                                d.get("cand_ids"), n_cands=n_c, cache=False)
            autotuned["small"] = {"best": list(best), "candidates": len(times), "best_ms": times[best],
                                  "ms": {",".join(map(str, k)): v for k, v in times.items()}}
        if args.autotune:
            best, times = tuning.autotune(d["points"], d["poly_offsets"], d["verts"], d.get("cand_offsets"),
                                          d.get("cand_ids"), n_cands=n_c, cache=False)
            autotuned["large"] = {"best": list(best), "candidates": len(times), "best_ms": times[best]}
        autotuned = autotuned or None
    fn = api.pip_classify if args.kernel == "filtered" else api.pip_classify_exact
    if args.semantics != "halfopen":
        algorithm = 1 if args.semantics == "alg1" else 2

        def fn(*a_, **k_):
            return api.pip_classify_paper(*a_, algorithm=algorithm, **k_)
    index_info = None
    if args.index == "slab":
        torch.cuda.synchronize()
        tb0 = time.perf_counter()
        slab = api.slab_index(d["poly_offsets"], d["verts"], args.edges_per_slab)
        torch.cuda.synchronize()
        build_ms = 1000 * (time.perf_counter() - tb0)
        index_info = {"kind": "y-slab edge index (out of method: changes the pair tests, not the bits)",
                      "edges_per_slab": args.edges_per_slab, "build_ms_host_timed": build_ms,
                      "index_bytes": int(slab.numel())}

        def fn(*a_, **k_):
            return api.pip_classify_slab(*a_, index=slab, **k_)
    cand_o, cand_i = d.get("cand_offsets"), d.get("cand_ids")

    def call():
        fn(d["points"], d["poly_offsets"], d["verts"], cand_o, cand_i, out=out)

    # a step is one replay of a CUDA graph holding one call (warm-up calls on the capture stream
    # first, so that the library's per-stream work list exists before capture)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            call()
    stream.synchronize()
    graph = None
    per_replay = 0
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        l0 = api.pip_launch_count()
        with torch.cuda.graph(graph, stream=stream):
            call()
        per_replay = api.pip_launch_count() - l0

    def step():
        if graph is not None:
            graph.replay()
        else:
            call()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # inputs that an L2 of 126 MB could hold (below 160 MB): the L2 is flushed (a 256 MB write)
    # between timed steps, outside the events, and the step time is the mean of the per-step
    # intervals
    flush = None
    if B < 160 * 10**6:
        flush = torch.empty(256 * 2**20, dtype=torch.uint8, device="cuda")
    launches0 = api.pip_launch_count()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            if flush is not None:
                flush.zero_()
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
    launches = api.pip_launch_count() - launches0 + per_replay * args.steps
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    per = [ev0[i].elapsed_time(ev1[i]) for i in range(args.steps)]
    total_ms = sum(per) if flush is not None else ev0[0].elapsed_time(ev1[-1])
    total_ms = max_over_ranks(dist, total_ms)
    T_all = sum_over_ranks(dist, T)
    C_all = sum_over_ranks(dist, w.n_candidates)
    ms_step = total_ms / args.steps
    kern_ms = statistics.mean(per)

    # the other kernel on the same batch (comparison), a short run
    other_fn = api.pip_classify_exact if args.kernel == "filtered" else api.pip_classify
    other_ms = None
    if rank == 0:
        for _ in range(3):
            other_fn(d["points"], d["poly_offsets"], d["verts"], cand_o, cand_i, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_o = max(5, min(200, args.steps))
        with torch.cuda.stream(stream):   # the calls run on the stream the events are recorded on
            e0.record(stream)
            for _ in range(n_o):
                other_fn(d["points"], d["poly_offsets"], d["verts"], cand_o, cand_i, out=out)
            e1.record(stream)
        torch.cuda.synchronize()
        other_ms = e0.elapsed_time(e1) / n_o

    # e2e: host buffers through the public API (pinned H2D of every input, D2H of the bits)
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(getattr(w, k)).pin_memory() for k in ("points", "poly_offsets", "verts")}
        if not w.dense:
            host["cand_offsets"] = torch.from_numpy(w.cand_offsets).pin_memory()
            host["cand_ids"] = torch.from_numpy(w.cand_ids).pin_memory()
        hout = torch.empty(n_words, dtype=torch.int32).pin_memory()
        h2d = sum(t_.numel() * t_.element_size() for t_ in host.values())
        d2h = hout.numel() * 4

        def e2e_step():
            for k_, v_ in host.items():
                d[k_].copy_(v_, non_blocking=True)
            fn(d["points"], d["poly_offsets"], d["verts"], d.get("cand_offsets"), d.get("cand_ids"), out=out)
            hout.copy_(out, non_blocking=True)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):   # copies and calls on the stream the events are recorded on
            e0.record(stream)
            for _ in range(args.e2e_steps):
                e2e_step()
            e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(dist, e0.elapsed_time(e1)) / args.e2e_steps
        e2e = {"value": job_rate(T_all, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms}

    peaks, peak_kind = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    achieved_gbs = B / (kern_ms / 1000.0) / 1e9
    small_name = SMALL_KERNEL_NAMES.get(api.pip_get_small_tuning()[0], "k_pip_warp")
    traffic = profiled_traffic(args.workload, small_name) if args.kernel == "filtered" and args.scale == 1.0 else None
    roof = roofline_of(T, B, kern_ms, peaks, peak_kind, n_sm,
                       f"{small_name} + k_pip_large" if args.kernel == "filtered" else "k_pip_exact", traffic)
    other_roof = None
    if other_ms:
        other_roof = roofline_of(T, B, other_ms, peaks, peak_kind, n_sm,
                                 "k_pip_exact" if args.kernel == "filtered" else f"{small_name} + k_pip_large")
        other_roof = {k: other_roof[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(w)
    verification = None
    if args.verify and args.kernel == "filtered" and args.semantics == "halfopen":
        api.pip_set_verify(True)
        try:
            api.pip_reset_stats()
            fn(d["points"], d["poly_offsets"], d["verts"], cand_o, cand_i, out=out)
            torch.cuda.synchronize()
            vs = api.pip_get_stats()
        finally:
            api.pip_set_verify(False)
        verification = {"filter_errors": vs["filter_errors"], "verified_pairs": vs["verified_pairs"]}
    semantics = None
    if args.semantics != "halfopen":
        # bits where the paper's printed rule and the half-open rule disagree (not timed)
        ref = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], cand_o, cand_i)
        fn(d["points"], d["poly_offsets"], d["verts"], cand_o, cand_i, out=out)
        x = torch.bitwise_xor(out[:n_words], ref[:n_words]).view(torch.uint8).cpu().numpy()
        diff = int(np.unpackbits(x).sum())
        semantics = {"rule": args.semantics, "bits_differing_from_half_open": diff,
                     "fraction_of_candidates": diff / max(1, w.n_candidates)}

    others = None
    if rank == 0:
        stats = api.pip_get_stats()
        if (world == 1 and args.workload == "footprints" and args.scale == 1.0 and not args.no_other_configs
                and args.kernel == "filtered" and args.semantics == "halfopen" and args.index == "none"):
            del d, out
            torch.cuda.empty_cache()
            others = other_configs(args, peaks, peak_kind, n_sm)
        line = {
            "metric": METRIC, "value": job_rate(T_all, ms_step), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": arithmetic_of(w) if args.kernel == "filtered" else "i64",
            "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.n_polys} polygons, {w.n_candidates} candidates, "
                                   f"{w.verts.shape[0]} vertices", "pair_tests_per_step": T,
                       "algorithmic_bytes_per_step": B, "kernel": args.kernel,
                       "tuning": list(api.pip_get_tuning()), "small_tuning": list(api.pip_get_small_tuning()),
                       "autotuned": autotuned,
                       "timing": "one CUDA-graph replay per step" if graph is not None else "direct calls",
                       "l2": ("L2 flushed between steps (256 MB write, outside the timed intervals)"
                              if flush is not None else "inputs larger than L2 (no flush)")},
            "points_per_s": job_rate(C_all, ms_step),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "other_kernel": {"kernel": "exact" if args.kernel == "filtered" else "filtered",
                             "ms_per_step": other_ms,
                             "value": (T / (other_ms / 1000.0)) if other_ms else None,
                             "roofline": other_roof},
            "fallback_fraction": (stats["fallback_points"] / stats["candidates"]) if stats["candidates"] else None,
            "wait_timeouts": stats["wait_timeouts"],
        }
        if others is not None:
            line["other_configs"] = others
        if verification is not None:
            line["verification"] = verification
        if index_info:
            line["metric"] = "points classified/s through a y-slab edge index (1 GB300), 0 mismatches"
            line["unit"] = "points/s"
            line["value"] = line["points_per_s"]
            line["index"] = index_info
            line["config"]["kernel"] = "k_pip_warp + k_pip_large (y-slab index)"
            line["method_pair_tests_per_s_equivalent"] = job_rate(T_all, ms_step)
            # the pair tests are no longer the method's T: report the bytes roofline instead
            line["roofline"] = {"bound": "hbm", "achieved": achieved_gbs, "peak": float(peaks["hbm_gbs"]),
                                "unit": "GB/s", "frac": achieved_gbs / float(peaks["hbm_gbs"]), "traffic": None,
                                "peak_source": peak_kind, "kernel": "k_pip_warp + k_pip_large (y-slab index)",
                                "algorithmic_bytes": B, "kernel_ms": kern_ms}
            line["e2e"] = None if e2e is None else dict(e2e, value=job_rate(C_all, e2e["ms_per_step"]), unit="points/s")
            line["cpu_baseline"] = None if cpu is None else dict(cpu, value=cpu["points_per_s"], unit="points/s")
        if semantics:
            line["semantics"] = semantics
            line["config"]["kernel"] = f"paper {args.semantics} (plain exact kernel)"
            line["roofline"]["kernel"] = "k_pip_exact (paper rule)"
            line["dtype"] = "i64" if args.semantics == "alg1" else "f64"
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
