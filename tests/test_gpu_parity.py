"""GPU parity: both kernels through the C ABI against the CPU oracle, bit for bit.

Every case below compares all output bits (0 mismatches required) unless it says
"sampled": at the full sizes whose oracle run would take minutes, a seeded sample of
candidates is checked one by one with the oracle's sampled entry point.
"""
import numpy as np
import pytest

import oracle
from paper_2306_04316_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_04316_gb300 import api as _api, build
    build.build_library()
    oracle.build()
    return _api


def gpu_bits(api, w, exact=False, dev="cuda"):
    d = api.to_device(w, dev)
    fn = api.pip_classify_exact if exact else api.pip_classify
    out = fn(d["points"], d["poly_offsets"], d["verts"], d.get("cand_offsets"), d.get("cand_ids"),
             n_cands=None if w.dense else w.n_bits)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)[:w.n_words]


def assert_same(got, want, n_bits, what):
    if not np.array_equal(got, want):
        g, o = oracle.unpack_bits(got, n_bits), oracle.unpack_bits(want, n_bits)
        bad = np.nonzero(g != o)[0]
        raise AssertionError(f"{what}: {len(bad)} mismatched bits of {n_bits}; first {bad[:10].tolist()}")


def check_full(api, w, what=""):
    want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
    for exact in (False, True):
        got = gpu_bits(api, w, exact)
        assert_same(got, want, w.n_bits, f"{w.name} {what} {'exact' if exact else 'filtered'}")


def make(name, polys, points, csr=None):
    """Workload from python lists: polys = list of vertex lists, csr = list of id lists."""
    po = np.zeros(len(polys) + 1, dtype=np.int64)
    po[1:] = np.cumsum([len(p) for p in polys])
    verts = np.array([v for p in polys for v in p], dtype=np.int64).reshape(-1, 2).astype(np.int32)
    pts = np.array(points, dtype=np.int64).reshape(-1, 2).astype(np.int32)
    w = W.Workload(name, pts, po.astype(np.int32), verts)
    if csr is not None:
        co = np.zeros(len(csr) + 1, dtype=np.int64)
        co[1:] = np.cumsum([len(c) for c in csr])
        ids = np.array([i for c in csr for i in c], dtype=np.int32)
        w = w.with_csr(co.astype(np.int32), ids)
    return w


# ------------------------------------------------------------------------------------------
# small and degenerate cases
# ------------------------------------------------------------------------------------------

def test_golden_cases(api):
    import json, os
    g = os.path.join(os.path.dirname(__file__), "golden")
    d = json.load(open(os.path.join(g, "diamond.json")))
    s = json.load(open(os.path.join(g, "square.json")))
    w = make("diamond", [d["verts"]], [d["point"]])
    for exact in (False, True):
        assert oracle.unpack_bits(gpu_bits(api, w, exact), 1)[0] == d["inside_half_open"]
    w = make("square", [s["verts"]], [c[0] for c in s["cases"]])
    want = np.array([c[1] for c in s["cases"]])
    for exact in (False, True):
        assert (oracle.unpack_bits(gpu_bits(api, w, exact), len(want)) == want).all()


@pytest.mark.parametrize("n_points", [0, 1, 31, 32, 33, 1000])
def test_point_counts_dense(api, n_points):
    rng = np.random.default_rng(n_points)
    polys = [[tuple(map(int, rng.integers(0, 40, 2))) for _ in range(int(rng.integers(3, 12)))] for _ in range(5)]
    pts = rng.integers(-2, 42, size=(n_points, 2))
    w = make("dense-small", polys, pts)
    if w.n_words == 0:
        return
    check_full(api, w)


def test_lattice_degeneracies(api):
    """Tiny lattice polygons with repeated vertices, collinear runs, horizontal edges,
    self-intersections and an explicit closing vertex; every lattice point of [-1, 17]^2."""
    rng = np.random.default_rng(5)
    polys = []
    for t in range(300):
        m = int(rng.integers(3, 9))
        v = [tuple(map(int, rng.integers(0, 17, 2))) for _ in range(m)]
        if t % 4 == 1:
            v = v[:2] + [v[1]] + v[2:]
        elif t % 4 == 2:
            v = v + [(int(rng.integers(0, 17)), v[-1][1])]
        elif t % 4 == 3:
            v = v + [v[0]]
        polys.append(v)
    xs, ys = np.meshgrid(np.arange(-1, 18), np.arange(-1, 18))
    pts = np.stack([xs.ravel(), ys.ravel()], 1)
    check_full(api, make("lattice", polys, pts))


def test_degenerate_polygons_and_empty_lists(api):
    rng = np.random.default_rng(6)
    polys = [[], [(1, 1)], [(0, 0), (5, 5)], [(0, 0), (4, 0), (0, 4)], [], [(0, 0), (9, 0), (9, 9), (0, 9)]]
    pts = rng.integers(-1, 11, size=(200, 2))
    csr = [list(range(0, 50)), [], list(range(10, 90)), list(range(200)), list(range(5)), list(range(199, -1, -1))]
    check_full(api, make("degenerate-csr", polys, pts, csr))
    check_full(api, make("degenerate-dense", polys, pts))


def test_int32_extremes(api):
    lo, hi = -2**31, 2**31 - 1
    polys = [[(lo, lo), (hi, lo), (hi, hi), (lo, hi)],
             [(lo, lo), (hi, hi), (lo, hi)],
             [(lo, 0), (0, lo), (hi, 0), (0, hi)],
             [(lo, lo), (hi, lo + 1), (lo + 2, hi)]]
    pts = [(lo, lo), (hi, hi), (lo, hi), (hi, lo), (0, 0), (lo + 1, lo), (hi - 1, hi - 1), (lo, 0), (hi, 0),
           (-1, -1), (1, 1), (lo + 1, lo + 1), (0, lo), (0, hi), (hi - 1, lo)]
    rng = np.random.default_rng(7)
    pts += [tuple(map(int, rng.integers(lo, hi, 2, endpoint=True))) for _ in range(400)]
    check_full(api, make("extremes", polys, pts))


def test_many_empty_polygons_in_one_chunk(api):
    """A chunk of candidates whose owning polygons are spread over more than one window of
    polygon offsets (hundreds of polygons with no candidates in between)."""
    rng = np.random.default_rng(8)
    polys, csr = [], []
    for k in range(3000):
        cx, cy = int(rng.integers(0, 10**6)), int(rng.integers(0, 10**6))
        m = int(rng.integers(3, 9))
        ang = np.sort(rng.uniform(0, 2 * np.pi, m))
        polys.append([(cx + int(300 * np.cos(a)), cy + int(300 * np.sin(a))) for a in ang])
        csr.append([] if k % 7 else list(rng.integers(0, 5000, int(rng.integers(0, 3)))))
    pts = rng.integers(0, 10**6, size=(5000, 2))
    for k in range(0, 3000, 7):   # give listed candidates a chance to be inside
        for j, pid in enumerate(csr[k]):
            pts[pid] = polys[k][0][0] - 10, polys[k][0][1]
    check_full(api, make("sparse-csr", polys, pts, csr))


@pytest.mark.parametrize("tuning", [(256, 1, 1), (512, 2, 2), (1024, 4, 2), (2048, 2, 4), (2048, 4, 3), (8192, 1, 1)])
def test_tuning_shapes(api, tuning):
    """Every tuned shape gives the same bits (small edge tiles force the streamed path)."""
    before = api.pip_get_tuning()
    api.pip_set_tuning(*tuning)
    try:
        w = W.footprints(seed=11, n_polys=4000, pts_per_poly=16)
        check_full(api, w, f"tuning={tuning}")
        big = W.fractal(seed=12, n_polys=4, m_lo=3000, m_hi=9000, n_points=30000, cell=200_000, grid=2)
        check_full(api, big, f"tuning={tuning}")
        s = W.star(seed=13, m=1024, n_uniform=4000, n_special=300)
        check_full(api, s, f"tuning={tuning}")
    finally:
        api.pip_set_tuning(*before)


# ------------------------------------------------------------------------------------------
# the five workloads
# ------------------------------------------------------------------------------------------

def test_star_full(api):
    w = W.star()
    check_full(api, w)


def test_footprints_reduced(api):
    check_full(api, W.footprints(n_polys=50_000))


def test_footprints_scattered_points(api):
    check_full(api, W.scattered_points(W.footprints(seed=21, n_polys=20_000)))


@pytest.mark.parametrize("kernel", [0, 1, 2], ids=["lockstep", "compacting", "thread-per-polygon"])
def test_filter_statistics(api, kernel):
    """The device counters of the filtered kernel, under each small-polygon kernel: every
    candidate is counted once, the box rejects equal a numpy count of candidates outside their
    polygon's closed bounding box, and the exact rechecks are a subset of the rest."""
    w = W.footprints(seed=5, n_polys=20_000)
    before = api.pip_get_small_tuning()
    api.pip_set_small_tuning(kernel, 0, -1)
    try:
        api.pip_reset_stats()
        gpu_bits(api, w)
        s = api.pip_get_stats()
    finally:
        api.pip_set_small_tuning(*before)
    po, v, co, ids = w.poly_offsets.astype(np.int64), w.verts, w.cand_offsets.astype(np.int64), w.cand_ids
    owner = np.repeat(np.arange(len(po) - 1), np.diff(co))
    lo = np.stack([np.minimum.reduceat(v[:, k], po[:-1]) for k in (0, 1)], 1)
    hi = np.stack([np.maximum.reduceat(v[:, k], po[:-1]) for k in (0, 1)], 1)
    p = w.points[ids]
    inside = np.all((p >= lo[owner]) & (p <= hi[owner]), axis=1)
    assert s["candidates"] == w.n_bits
    assert s["bbox_rejects"] == int((~inside).sum())
    assert 0 <= s["fallback_points"] <= int(inside.sum())


def test_stress_reduced(api):
    check_full(api, W.stress(n_polys=60_000))


def test_fractal_reduced(api):
    w = W.fractal(n_polys=6, m_lo=5_000, m_hi=40_000, n_points=150_000, cell=400_000, grid=3)
    check_full(api, w)


def test_join_reduced(api):
    """Binning then classification: the GPU candidate sets equal the oracle's closed-bbox sets
    polygon by polygon, and classification of that CSR matches the oracle."""
    w = W.join(n_polys=3000, n_points=300_000)
    d = api.to_device(w)
    co, ids = api.bin_join(d["points"], d["poly_offsets"], d["verts"])
    torch.cuda.synchronize()
    co = co.cpu().numpy()
    ids = ids.cpu().numpy()
    counts, want_ids = oracle.bbox_join(w.points, w.poly_offsets, w.verts, np.arange(w.n_polys))
    assert np.array_equal(np.diff(co.astype(np.int64)), counts)
    pos = 0
    for k in range(w.n_polys):
        a = np.sort(ids[co[k]:co[k + 1]])
        assert np.array_equal(a, want_ids[pos:pos + counts[k]]), f"polygon {k}"
        pos += counts[k]
    # classification parity on the oracle's own candidate lists (no oracle input from the GPU)
    oco = np.zeros(w.n_polys + 1, dtype=np.int64)
    oco[1:] = np.cumsum(counts)
    check_full(api, w.with_csr(oco, want_ids), "joined")


def test_binning_is_deterministic(api):
    w = W.join(seed=31, n_polys=2000, n_points=200_000)
    d = api.to_device(w)
    co1, ids1 = api.bin_join(d["points"], d["poly_offsets"], d["verts"])
    co2, ids2 = api.bin_join(d["points"], d["poly_offsets"], d["verts"])
    torch.cuda.synchronize()
    assert torch.equal(co1, co2) and torch.equal(ids1, ids2)


@pytest.mark.parametrize("exact", [False, True])
def test_out_of_range_ids_read_nothing(api, exact):
    """Candidate ids outside [0, n_points) are never dereferenced: their bits are 0 and every
    valid candidate keeps its oracle bit, for small polygons and for a large one."""
    rng = np.random.default_rng(5)
    small = make("small", [[(0, 0), (100, 0), (100, 100), (0, 100)]] * 3, rng.integers(-10, 110, (500, 2)),
                 csr=[range(500)] * 3)
    big = make("big", [_star_polygon(rng, 600, 50_000)], rng.integers(-60_000, 60_000, (3000, 2)),
               csr=[range(3000)])
    w = _concat([small, big], "mixed")
    ids = w.cand_ids.copy()
    bad = rng.choice(len(ids), 200, replace=False)
    ids[bad[:100]] = -1 - rng.integers(0, 2**31 - 1, 100)
    ids[bad[100:]] = w.n_points + rng.integers(0, 2**31 - 1 - w.n_points, 100)
    got = oracle.unpack_bits(gpu_bits(api, w.with_csr(w.cand_offsets, ids.astype(np.int32)), exact=exact),
                             w.n_bits)
    want = oracle.unpack_bits(oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids),
                              w.n_bits)
    keep = np.ones(w.n_bits, bool)
    keep[bad] = False
    assert not got[bad].any()
    assert np.array_equal(got[keep], want[keep])


def _bin_case(rng):
    """Polygons that exercise every path of the binning: tiny boxes, boxes large enough to go on
    the short list, empty polygons, and id lists long enough for each sort (a lane's registers,
    a warp's registers at 1, 2 and 4 ids a lane, warp shared memory, CTA shared memory, global
    memory)."""
    polys = []
    for _ in range(300):                      # tiny squares (a few points each)
        x, y = rng.integers(-10**6, 10**6, 2)
        s = int(rng.integers(50, 400))
        polys.append(np.array([[x, y], [x + s, y], [x + s, y + s], [x, y + s]], dtype=np.int64))
    hot = rng.integers(-10**6 + 50_000, 10**6 - 50_000, (2, 2))          # two hot spots of points
    for (x, y), s in zip(hot, (3000, 16000)):                            # ~10^2 and ~10^3 points
        polys.append(np.array([[x, y], [x + s, y], [x, y + s]], dtype=np.int64))
    x, y = hot[0] - 19_000                    # lists of about 20, 50, 100, 400 and 850 ids
    for s in (1500, 2300, 3300, 6500, 9500):
        polys.append(np.array([[x, y], [x + s, y], [x, y + s]], dtype=np.int64))
    polys.append(np.zeros((0, 2), dtype=np.int64))                      # empty polygon
    big = 2 * 10**6
    polys.append(np.array([[-big, -big], [big, -big], [0, big]], dtype=np.int64))   # covers everything
    for i in range(300):                      # many wide, flat boxes: the short list fills up
        y = -10**6 + 6000 * i
        polys.append(np.array([[-10**6, y], [10**6, y], [0, y + 40]], dtype=np.int64))
    po = np.zeros(len(polys) + 1, dtype=np.int64)
    po[1:] = np.cumsum([len(q) for q in polys])
    verts = np.concatenate(polys).astype(np.int32)
    pts = rng.integers(-10**6, 10**6, (300_000, 2)).astype(np.int32)
    extra = [(c + rng.integers(-20_000, 20_000, (30_000, 2))) for c in hot]
    pts = np.concatenate([pts] + [e.astype(np.int32) for e in extra])
    return pts, po.astype(np.int32), verts


@pytest.mark.parametrize("cell_size", [0, 1, 1 << 12, 1 << 20])
def test_binning_paths_and_cell_sizes(api, cell_size):
    """Every candidate list equals the oracle's closed-box list exactly (ids ascending), for the
    automatic cell size and for requested ones from one unit (raised to what the pair list
    holds) to a quarter of the domain."""
    rng = np.random.default_rng(77)
    pts, po, verts = _bin_case(rng)
    P = len(po) - 1
    d_pts, d_po, d_v = (torch.from_numpy(x).cuda() for x in (pts, po, verts))
    co, ids = api.bin_join(d_pts, d_po, d_v, cell_size=cell_size)
    torch.cuda.synchronize()
    counts, want_ids = oracle.bbox_join(pts, po, verts, np.arange(P))
    assert counts.max() > 8192
    for lo, hi in ((1, 16), (16, 32), (32, 64), (64, 128), (128, 512), (512, 8192)):
        assert ((counts > lo) & (counts <= hi)).any(), (lo, hi)
    assert np.array_equal(np.diff(co.cpu().numpy().astype(np.int64)), counts)
    assert np.array_equal(ids.cpu().numpy(), want_ids)


def test_binning_degenerate_inputs(api):
    """Empty point sets and polygon sets, boxes of zero width or height, points exactly on box
    edges and corners (closed boxes include them), and more (polygon, point) pairs than the
    probe workspace records (the fill pass then probes the points again): every list equals
    the oracle's."""
    rng = np.random.default_rng(79)
    polys = [np.array([[0, 0], [0, 1000], [0, 500]], dtype=np.int64),          # zero width
             np.array([[0, 0], [1000, 0], [500, 0]], dtype=np.int64),          # zero height
             np.array([[5, 5]], dtype=np.int64),                                # a single vertex
             np.array([[-100, -100], [100, -100], [100, 100], [-100, 100]], dtype=np.int64)]
    polys += [np.array([[-50 - i, -50], [50, -50 - i], [50 + i, 50], [-50, 50 + i]], dtype=np.int64)
              for i in range(600)]                                             # 600 overlapping boxes
    po = np.zeros(len(polys) + 1, dtype=np.int64)
    po[1:] = np.cumsum([len(q) for q in polys])
    verts = np.concatenate(polys).astype(np.int32)
    edge_pts = [(0, 0), (0, 1000), (0, 500), (1000, 0), (500, 0), (5, 5), (-100, -100), (100, 100),
                (-100, 100), (100, -100), (0, 1001), (1001, 0), (-101, 0)]
    pts = np.concatenate([np.array(edge_pts), rng.integers(-120, 120, (2000, 2))]).astype(np.int32)
    P = len(po) - 1
    d_po, d_v = torch.from_numpy(po.astype(np.int32)).cuda(), torch.from_numpy(verts).cuda()
    for case_pts in (pts, pts[:0]):
        d_pts = torch.from_numpy(np.ascontiguousarray(case_pts)).cuda()
        co, ids = api.bin_join(d_pts, d_po, d_v)
        torch.cuda.synchronize()
        counts, want_ids = oracle.bbox_join(case_pts, po.astype(np.int32), verts, np.arange(P))
        if len(case_pts):
            assert counts.sum() > len(case_pts) // 2 + 1024        # past what the probe records
        assert np.array_equal(np.diff(co.cpu().numpy().astype(np.int64)), counts)
        assert np.array_equal(ids.cpu().numpy(), want_ids)
    # no polygons at all
    e_po = torch.zeros(1, dtype=torch.int32, device="cuda")
    e_v = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    co, ids = api.bin_join(torch.from_numpy(pts).cuda(), e_po, e_v)
    torch.cuda.synchronize()
    assert co.cpu().tolist() == [0] and ids.numel() == 0


def test_binning_index_probed_by_several_batches(api):
    """One polygon index, three batches of points probed on two streams at once (each with its
    own probe workspace): every batch's CSR equals the oracle's; an index built for another
    polygon count, or never built, yields no candidates."""
    rng = np.random.default_rng(78)
    pts0, po, verts = _bin_case(rng)
    P = len(po) - 1
    d_po, d_v = torch.from_numpy(po).cuda(), torch.from_numpy(verts).cuda()
    index = api.bin_index(d_po, d_v)
    batches = [pts0, rng.permutation(pts0)[:200_000], rng.integers(-10**6, 10**6, (50_000, 2)).astype(np.int32)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    out = []
    for b, pts in enumerate(batches):
        st = streams[b % 2]
        d_pts = torch.from_numpy(pts).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            co, tot, probe = api.pip_bin_probe_count(d_pts, index, P, stream=st)
            st.synchronize()
            ids = torch.empty(max(int(tot.item()), 1), dtype=torch.int32, device="cuda")
            ovf = torch.zeros(1, dtype=torch.int32, device="cuda")
            api.pip_bin_probe_fill(d_pts, index, P, probe, co, ids, d_overflow=ovf, stream=st)
        out.append((co, tot, ids, ovf, pts))
    torch.cuda.synchronize()
    for co, tot, ids, ovf, pts in out:
        counts, want_ids = oracle.bbox_join(pts, po, verts, np.arange(P))
        assert int(ovf.item()) == 0 and int(tot.item()) == counts.sum()
        assert np.array_equal(np.diff(co.cpu().numpy().astype(np.int64)), counts)
        assert np.array_equal(ids[:int(tot.item())].cpu().numpy(), want_ids)
    d_pts = torch.from_numpy(pts0).cuda()
    co, tot, _ = api.pip_bin_probe_count(d_pts, index, P - 1)             # another polygon count
    fresh = torch.zeros_like(index)                                        # never built
    co2, tot2, _ = api.pip_bin_probe_count(d_pts, fresh, P)
    torch.cuda.synchronize()
    assert int(tot.item()) == 0 and not co.any()
    assert int(tot2.item()) == 0 and not co2.any()


def _concat(ws, name):
    """Concatenate CSR workloads (polygons, points and candidate lists) into one."""
    pts, po, vs, co, ids = [], [0], [], [0], []
    npts = nv = nc = 0
    for w in ws:
        pts.append(w.points)
        vs.append(w.verts)
        po += list(np.asarray(w.poly_offsets[1:], dtype=np.int64) + nv)
        co += list(np.asarray(w.cand_offsets[1:], dtype=np.int64) + nc)
        ids.append(w.cand_ids.astype(np.int64) + npts)
        npts += w.n_points
        nv += w.verts.shape[0]
        nc += w.n_bits
    return W.Workload(name, np.concatenate(pts), np.array(po, dtype=np.int32), np.concatenate(vs),
                      np.array(co, dtype=np.int32), np.concatenate(ids).astype(np.int32))


def test_small_and_large_polygons_interleaved(api):
    """Output words shared by small polygons (batched kernel) and large ones (large-polygon
    kernel, XOR into the same words); candidate blocks not aligned to words."""
    parts = []
    for i in range(6):
        parts.append(W.footprints(seed=100 + i, n_polys=37 + 5 * i, pts_per_poly=3 + i))
        parts.append(W.fractal(seed=200 + i, n_polys=1, m_lo=121 + 400 * i, m_hi=122 + 400 * i,
                               n_points=700 + 131 * i, cell=100_000, grid=1))
    check_full(api, _concat(parts, "mixed"))


def test_large_list_overflow_scan_mode(api):
    """More large polygons than the per-call list holds (65,536): the large-polygon kernel
    falls back to scanning every polygon."""
    rng = np.random.default_rng(41)
    n = 66_000
    m = 124
    ang = np.sort(rng.uniform(0, 2 * np.pi, (n, m)), axis=1)
    cx = rng.integers(-10**9, 10**9, n)[:, None]
    cy = rng.integers(-10**9, 10**9, n)[:, None]
    vx = (cx + 1000 * np.cos(ang)).astype(np.int64)
    vy = (cy + 1000 * np.sin(ang)).astype(np.int64)
    verts = np.stack([vx.ravel(), vy.ravel()], 1).astype(np.int32)
    po = (np.arange(n + 1) * m).astype(np.int32)
    pts = np.stack([np.concatenate([cx[:, 0], cx[:, 0] + 990]), np.concatenate([cy[:, 0], cy[:, 0]])], 1)
    co = (np.arange(n + 1) * 2).astype(np.int32)
    ids = np.stack([np.arange(n), np.arange(n) + n], 1).ravel().astype(np.int32)
    w = W.Workload("overflow", pts.astype(np.int32), po, verts, co, ids)
    check_full(api, w)


def test_repeated_calls_and_streams(api):
    """The large-polygon list empties itself: repeated calls, and calls on a second stream."""
    w = W.fractal(seed=51, n_polys=3, m_lo=2000, m_hi=5000, n_points=20_000, cell=300_000, grid=2)
    want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
    d = api.to_device(w)
    s2 = torch.cuda.Stream()
    for i in range(4):
        st = s2 if i % 2 else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            out = api.pip_classify(d["points"], d["poly_offsets"], d["verts"], d["cand_offsets"], d["cand_ids"],
                                   n_cands=w.n_bits)
        st.synchronize()
        assert_same(out.cpu().numpy().view(np.uint32)[:w.n_words], want, w.n_bits, f"call {i}")


def test_full_range_boxes_points_on_extremes(api):
    """Polygons whose box spans the whole int32 range (P - o reaches 2^31) with points on the
    extreme rows and columns, in CSR and dense mode."""
    lo, hi = -2**31, 2**31 - 1
    polys = [[(lo, lo), (hi, lo), (hi, hi)], [(lo, lo), (hi, hi), (lo, hi)], [(hi, lo), (hi, hi), (lo, 0)],
             [(lo, lo), (hi, 0), (lo, hi)], [(lo, 0), (0, lo), (hi, 0), (0, hi)],
             [(lo, lo), (hi, lo), (hi, hi), (lo, hi)]]
    rng = np.random.default_rng(71)
    pts = []
    for _ in range(300):
        t = int(rng.integers(lo, hi, endpoint=True))
        pts += [(hi, t), (lo, t), (t, hi), (t, lo), (hi - 1, t), (lo + 1, t)]
    pts += [(hi, hi), (lo, lo), (hi, lo), (lo, hi), (hi, 0), (0, hi), (-1, -1), (0, 0)]
    ids = list(range(len(pts)))
    check_full(api, make("full-range-csr", polys, pts, [ids] * len(polys)))
    check_full(api, make("full-range-dense", polys, pts))


def _star_polygon(rng, m, radius, centre=(0, 0)):
    ang = np.sort(rng.uniform(0, 2 * np.pi, m))
    rad = rng.uniform(0.5, 1.0, m) * radius
    v = np.stack([centre[0] + rad * np.cos(ang), centre[1] + rad * np.sin(ang)], 1)
    return np.clip(np.rint(v), -2**31, 2**31 - 1).astype(np.int64)


def test_large_polygons_full_range_and_near_the_frame_limit(api):
    """Large-polygon kernel tiles whose frame reaches 2^30 from its centre or more (int64 and
    double records, edge-by-edge bounds) and tiles just below that limit (scaled records, the
    sign-bit straddle test); points uniform, on vertices, on edge midpoints and at the extremes."""
    rng = np.random.default_rng(2306043160 + 81)
    polys = [_star_polygon(rng, 2000, 2.0**31), _star_polygon(rng, 1500, 2.0**29.95),
             _star_polygon(rng, 700, 2.0**30.2, centre=(2.0**30, -2.0**30))]
    pts = [rng.integers(-2**31, 2**31, (3000, 2), endpoint=False)]
    for v in polys:
        pts.append(v[rng.integers(0, len(v), 200)])
        a, b = v, np.roll(v, -1, axis=0)
        even = ((a + b) % 2 == 0).all(axis=1)
        pts.append(((a + b) // 2)[even][:200])
    lo, hi = -2**31, 2**31 - 1
    pts.append(np.array([(lo, lo), (hi, hi), (lo, hi), (hi, lo), (0, 0), (hi, 0), (0, lo)]))
    pts = np.concatenate(pts).astype(np.int64)
    w = make("large-full-range", [v.tolist() for v in polys], pts.tolist())
    check_full(api, w)
    api.pip_set_verify(True)
    try:
        api.pip_reset_stats()
        got = gpu_bits(api, w)
        s = api.pip_get_stats()
    finally:
        api.pip_set_verify(False)
    assert_same(got, oracle.classify(w.points, w.poly_offsets, w.verts), w.n_bits, "verification mode")
    assert s["verified_pairs"] > 0 and s["filter_errors"] == 0 and s["wait_timeouts"] == 0


# ------------------------------------------------------------------------------------------
# soundness of the fast paths (verification mode)
# ------------------------------------------------------------------------------------------

def _verify_cases():
    return [
        ("footprints", lambda: W.footprints(seed=9, n_polys=20_000)),          # int32 path
        ("stress", lambda: W.stress(seed=10, n_polys=40_000)),                 # FP32 filter, full range
        ("star", lambda: W.star()),                                           # large-polygon kernel
        ("fractal", lambda: W.fractal(seed=11, n_polys=4, m_lo=3_000, m_hi=20_000, n_points=60_000,
                                      cell=300_000, grid=2)),
    ]


@pytest.mark.parametrize("name,make_w", _verify_cases(), ids=[c[0] for c in _verify_cases()])
def test_verification_mode_finds_no_unsound_decision(api, name, make_w):
    """Every straddling pair whose fast-path decision the kernels trust (the int32 sign, or an
    FP32 sign outside the forward-error bound) is recomputed exactly: no disagreement, and the
    bits still equal the oracle's."""
    w = make_w()
    want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
    api.pip_set_verify(True)
    try:
        api.pip_reset_stats()
        got = gpu_bits(api, w)
        s = api.pip_get_stats()
    finally:
        api.pip_set_verify(False)
    assert_same(got, want, w.n_bits, f"{name} (verification mode)")
    assert s["verified_pairs"] > 0
    assert s["filter_errors"] == 0, f"{s['filter_errors']} of {s['verified_pairs']} trusted decisions were wrong"
    assert s["wait_timeouts"] == 0


@pytest.mark.parametrize("kernel", [0, 1, 2], ids=["lockstep", "compacting", "thread-per-polygon"])
def test_verification_mode_every_small_kernel(api, kernel):
    """Verification mode under each small-polygon kernel, on the footprint batch and on the
    int32-limit case (boxes at the corners of the int32 range against points anywhere in it, boxes
    at the int32 test's bound).  For the thread-per-polygon kernel this checks its clamp edge by
    edge: the int32 sign it computes on the clamped point must equal the exact sign on the raw
    point for every straddling pair of an in-bound polygon."""
    before = api.pip_get_small_tuning()
    api.pip_set_small_tuning(kernel, 0, -1)
    api.pip_set_verify(True)
    try:
        for w in (W.footprints(seed=9, n_polys=20_000), _extreme_small_case(np.random.default_rng(61))):
            want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
            api.pip_reset_stats()
            got = gpu_bits(api, w)
            s = api.pip_get_stats()
            assert_same(got, want, w.n_bits, f"{w.name} kernel {kernel} (verification mode)")
            assert s["verified_pairs"] > 0
            assert s["filter_errors"] == 0, f"{w.name}: {s['filter_errors']} of {s['verified_pairs']} wrong"
    finally:
        api.pip_set_verify(False)
        api.pip_set_small_tuning(*before)


# ------------------------------------------------------------------------------------------
# the paper's printed rules (pip_classify_paper)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("algorithm", [1, 2])
def test_paper_rules_match_the_oracle(api, algorithm):
    for w in (W.star(), W.stress(seed=12, n_polys=30_000)):
        d = api.to_device(w)
        out = api.pip_classify_paper(d["points"], d["poly_offsets"], d["verts"], d.get("cand_offsets"),
                                     d.get("cand_ids"), algorithm=algorithm,
                                     n_cands=None if w.dense else w.n_bits)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)[:w.n_words]
        want = oracle.classify_rule(w.points, w.poly_offsets, w.verts, algorithm, w.cand_offsets, w.cand_ids)
        assert_same(got, want, w.n_bits, f"{w.name} algorithm {algorithm}")


# ------------------------------------------------------------------------------------------
# CUDA-graph capture and replay (binning + classification)
# ------------------------------------------------------------------------------------------

def test_graph_replay_of_binning_and_classification(api):
    """One captured graph bins a batch of points and classifies it; replaying it after new
    points are copied into the same buffer gives each batch's oracle bits."""
    clusters, po, v = W.join_polygons(seed=2306043160 + 90, n_polys=2000)
    batches = [W.join_points(clusters, 2306043160 + 91 + b, 200_000) for b in range(3)]
    d_po, d_v = torch.from_numpy(po).cuda(), torch.from_numpy(v).cuda()
    d_pts = torch.from_numpy(batches[0]).cuda()
    P, n = len(po) - 1, len(batches[0])
    stream = torch.cuda.Stream()
    ws = api.bin_workspace(n, P)
    co = torch.empty(P + 1, dtype=torch.int32, device="cuda")
    tot = torch.empty(1, dtype=torch.int64, device="cuda")
    cap = 4 * n
    ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    out = torch.empty(cap // 32 + 1, dtype=torch.int32, device="cuda")
    ovf = torch.zeros(1, dtype=torch.int32, device="cuda")

    def step():
        api.pip_bin_count(d_pts, d_po, d_v, workspace=ws, cand_offsets=co, d_total=tot, stream=stream)
        api.pip_bin_fill(d_pts, d_po, d_v, ws, co, ids, d_overflow=ovf, stream=stream)
        api.pip_classify(d_pts, d_po, d_v, co, ids, out=out, stream=stream)

    with torch.cuda.stream(stream):
        step()                                   # first call on the stream: allocates its list
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step()
    for b in batches:
        d_pts.copy_(torch.from_numpy(b))
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            g.replay()
        stream.synchronize()
        assert int(ovf.item()) == 0
        n_c = int(tot.item())
        c_host = co.cpu().numpy().astype(np.int64)
        i_host = ids[:n_c].cpu().numpy()
        got = out.cpu().numpy().view(np.uint32)[:(n_c + 31) // 32]
        # candidate sets against the oracle's closed-box join; the bits against the oracle's
        # classification of its own candidate lists, matched by (polygon, point id)
        counts, want_ids = oracle.bbox_join(b, po, v, np.arange(P))
        assert np.array_equal(np.diff(c_host), counts)
        owner = np.repeat(np.arange(P), counts)
        perm = np.lexsort((i_host, owner))           # GPU positions in (polygon, id) order
        assert np.array_equal(i_host[perm], want_ids)
        oco = np.zeros(P + 1, dtype=np.int64)
        oco[1:] = np.cumsum(counts)
        want_bits = oracle.unpack_bits(oracle.classify(b, po, v, oco, want_ids), n_c)
        got_bits = oracle.unpack_bits(got, n_c)[perm]
        bad = np.nonzero(got_bits != want_bits)[0]
        assert len(bad) == 0, f"graph replay: {len(bad)} of {n_c} bits differ"


def _small_kernel_cases():
    """Workloads that exercise the small-polygon kernels' slicing: one slice per polygon set and
    several (more candidates than a slice), polygons with no candidates, sets cut by the vertex
    budget, dense small polygons whose slices span several polygons, int64/FP32 sets, large
    polygons interleaved with small ones, and invalid ids."""
    rng = np.random.default_rng(61)
    cases = [W.footprints(seed=62, n_polys=3000, pts_per_poly=16),
             W.footprints(seed=63, n_polys=300, pts_per_poly=700),
             W.footprints(seed=64, n_polys=5000, pts_per_poly=1),
             W.stress(seed=65, n_polys=4000)]
    # many polygons without candidates between listed ones
    polys, csr = [], []
    for k in range(2000):
        cx, cy = int(rng.integers(0, 10**6)), int(rng.integers(0, 10**6))
        m = int(rng.integers(3, 60))
        ang = np.sort(rng.uniform(0, 2 * np.pi, m))
        polys.append([(cx + int(300 * np.cos(a)), cy + int(300 * np.sin(a))) for a in ang])
        csr.append([] if k % 5 else [int(x) for x in rng.integers(0, 4000, int(rng.integers(1, 90)))])
    pts = rng.integers(0, 10**6, size=(4000, 2))
    for k in range(0, 2000, 5):
        for pid in csr[k]:
            pts[pid] = polys[k][0][0] - int(rng.integers(0, 400)), polys[k][0][1] + int(rng.integers(-200, 200))
    cases.append(make("sparse-sets", polys, pts, csr))
    # polygons of 200-256 vertices: every slice holds one polygon
    polys = [[(int(5000 * k + 2000 * np.cos(a)), int(3000 * np.sin(a)))
              for a in np.sort(rng.uniform(0, 2 * np.pi, int(rng.integers(200, 257))))] for k in range(60)]
    pts = [(int(5000 * k + x), int(y)) for k in range(60) for x, y in rng.integers(-2200, 2200, (40, 2))]
    cases.append(make("vertex-budget", polys, pts, [list(range(40 * k, 40 * k + 40)) for k in range(60)]))
    # dense: 300 small polygons against 100 points (slices span several polygons' candidates)
    polys = [[(int(50 * np.cos(a)) + int(rng.integers(-20, 20)), int(50 * np.sin(a)) + int(rng.integers(-20, 20)))
              for a in np.sort(rng.uniform(0, 2 * np.pi, int(rng.integers(3, 12))))] for _ in range(300)]
    cases.append(make("dense-small", polys, rng.integers(-60, 60, (100, 2))))
    # small and large interleaved
    parts = []
    for i in range(3):
        parts.append(W.footprints(seed=66 + i, n_polys=90 + 7 * i, pts_per_poly=5 + 3 * i))
        parts.append(W.fractal(seed=70 + i, n_polys=1, m_lo=300 + 500 * i, m_hi=301 + 500 * i,
                               n_points=900 + 77 * i, cell=100_000, grid=1))
    cases.append(_concat(parts, "interleaved"))
    cases.append(_extreme_small_case(rng))
    return cases


def _extreme_small_case(rng):
    """Small polygons whose pair tests sit at the limits of the 32-bit arithmetic: boxes at the
    corners of the int32 range against points anywhere in it (differences that wrap), boxes with
    (W + 1)(H + 1) exactly 2^30 and just above (the int32 test's bound), thin boxes of width about
    2^29, and polygons of 0, 1 and 2 vertices; candidates on vertices, edges and box sides."""
    I0, I1 = -2**31, 2**31 - 1
    polys, csr, pts = [], [], []

    def add(poly, extra):
        ids = []
        xs = [v[0] for v in poly] or [0]
        ys = [v[1] for v in poly] or [0]
        near = [(int(np.clip(x, I0, I1)), int(np.clip(y, I0, I1))) for x, y in zip(
            rng.integers(min(xs) - 3, max(xs) + 4, 24), rng.integers(min(ys) - 3, max(ys) + 4, 24))]
        for q in list(poly) + near + extra + [pts[int(i)] for i in rng.integers(0, max(1, len(pts)), 6) if pts]:
            ids.append(len(pts))
            pts.append(q)
        polys.append(poly)
        csr.append(ids)

    far = [tuple(int(c) for c in q) for q in rng.integers(I0, I1, (40, 2), endpoint=True)]
    for cx, cy in [(I0, I0), (I0, I1 - 40), (I1 - 40, I0), (I1 - 40, I1 - 40)]:
        for _ in range(6):
            m = int(rng.integers(3, 12))
            add([(cx + int(rng.integers(0, 41)), cy + int(rng.integers(0, 41))) for _ in range(m)], far)
    for w1, h1 in [(2**15, 2**15), (2**15 + 1, 2**15), (2**29, 2), (2**29 + 1, 2), (2**30, 1), (1, 2**30)]:
        W_, H_ = w1 - 1, h1 - 1
        x0, y0 = int(rng.integers(-2**30, 2**29)), int(rng.integers(-2**30, 2**29))
        poly = [(x0, y0), (x0 + W_ // 2, y0 + H_ // 3), (x0 + W_, y0), (x0 + W_, y0 + H_), (x0 + W_ // 3, y0 + H_ // 2),
                (x0, y0 + H_)]
        add(poly, [(x0 + W_ // 2, y0 + H_ // 2), (x0 - 1, y0 + H_ // 2), (x0 + W_ + 1, y0 + H_ // 2)] + far[:10])
    for m in (0, 1, 2, 0, 2, 1):
        add([(int(rng.integers(-50, 50)), int(rng.integers(-50, 50))) for _ in range(m)], far[:5])
    return make("extremes", polys, pts, csr)


@pytest.mark.parametrize("small", [(0, 256, 0), (0, 128, 0), (0, 256, 3), (1, 256, 0), (1, 128, 0), (1, 256, 1),
                                   (1, 128, 2), (2, 256, 0), (2, 128, 0), (2, 256, 1), (2, 128, 3)],
                         ids=lambda s: "k%d-%d-%d" % s)
def test_small_kernel_shapes(api, small):
    """Every small-polygon kernel, slice size (candidates per thread) and CTA count gives the
    oracle's bits."""
    before = api.pip_get_small_tuning()
    api.pip_set_small_tuning(*small)
    try:
        for w in _small_kernel_cases():
            want = oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids)
            assert_same(gpu_bits(api, w), want, w.n_bits, f"{w.name} small={small}")
        # invalid ids are never dereferenced
        w = W.footprints(seed=75, n_polys=2000, pts_per_poly=16)
        ids = w.cand_ids.copy()
        bad = np.random.default_rng(76).choice(len(ids), 300, replace=False)
        ids[bad[:150]] = -5
        ids[bad[150:]] = w.n_points + 7
        got = oracle.unpack_bits(gpu_bits(api, w.with_csr(w.cand_offsets, ids)), w.n_bits)
        want = oracle.unpack_bits(oracle.classify(w.points, w.poly_offsets, w.verts, w.cand_offsets, w.cand_ids),
                                  w.n_bits)
        keep = np.ones(w.n_bits, bool)
        keep[bad] = False
        assert not got[bad].any() and np.array_equal(got[keep], want[keep])
    finally:
        api.pip_set_small_tuning(*before)
