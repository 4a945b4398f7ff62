"""The JSON line of bench.py's reference arm (the oracle on the host's cores), run on CPU: one line
with the keys every bench line carries, the oracle described as the CPU baseline, and an
end-to-end figure equal to the line's own value (the oracle reads host memory, no copies)."""
import argparse
import io
import json
from contextlib import redirect_stdout

import bench


def test_reference_arm_line():
    args = argparse.Namespace(workload="footprints", steps=1, warmup=3)
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args, rank=0, world=1) == 0
    lines = [x for x in buf.getvalue().splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("footprints") and d["config"]["pair_tests_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
