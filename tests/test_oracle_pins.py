"""Pins of the CPU oracle (P1-P9): closed forms, brute force, invariants, golden cases."""
import pytest

import oracle
import pin_suite


@pytest.fixture(scope="module")
def lib():
    oracle.build()
    return oracle._load()


@pytest.mark.parametrize("pin", pin_suite.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(lib, pin):
    failures = pin(lib)
    assert not failures, "\n".join(failures)


def test_diamond_documents_literal_rule():
    """The paper's rule read literally counts the pass-through vertices twice (Method,
    steps 3-4 with Algorithm 1's <= 0): two crossings, 'outside' at the centre."""
    import json, os
    import pins
    d = json.load(open(os.path.join(pin_suite.GOLDEN, "diamond.json")))
    assert pins.literal_paper_count(*d["point"], d["verts"]) == d["literal_rule_crossings"]
    assert oracle.pip_single(*d["point"], d["verts"]) == d["inside_half_open"]


def test_sample_matches_full(lib):
    import numpy as np
    rng = np.random.default_rng(11)
    verts = rng.integers(-50, 50, size=(40, 2))
    po = np.array([0, 7, 7, 19, 40])
    pts = rng.integers(-55, 55, size=(300, 2))
    co = np.array([0, 100, 100, 250, 400])
    ids = rng.integers(0, 300, size=400)
    full = oracle.unpack_bits(oracle.classify(pts, po, verts, co, ids), 400)
    s = rng.choice(400, 60, replace=False)
    assert (oracle.classify_sample(pts, po, verts, s, co, ids) == full[s]).all()
    dense = oracle.unpack_bits(oracle.classify(pts, po, verts), 4 * 320)
    s = rng.choice(4 * 320, 80, replace=False)
    assert (oracle.classify_sample(pts, po, verts, s) == dense[s]).all()


def test_bbox_join_bruteforce(lib):
    import numpy as np
    rng = np.random.default_rng(12)
    verts = rng.integers(0, 100, size=(30, 2))
    po = np.array([0, 5, 12, 12, 30])
    pts = rng.integers(-5, 105, size=(500, 2))
    counts, ids = oracle.bbox_join(pts, po, verts, [0, 1, 2, 3])
    pos = 0
    for s, k in enumerate([0, 1, 2, 3]):
        v = verts[po[k]:po[k + 1]]
        if len(v) == 0:
            want = np.zeros(0, dtype=np.int64)
        else:
            m = (pts[:, 0] >= v[:, 0].min()) & (pts[:, 0] <= v[:, 0].max()) & \
                (pts[:, 1] >= v[:, 1].min()) & (pts[:, 1] <= v[:, 1].max())
            want = np.nonzero(m)[0]
        assert counts[s] == len(want)
        assert (ids[pos:pos + counts[s]] == want).all()
        pos += counts[s]
