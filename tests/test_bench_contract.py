"""bench.py on the host: the reference arm (the FP64 oracle on the host
cores) prints one JSON line with the keys its consumers read, and every
workload the bench offers builds and describes itself."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "cfg1",
           "--steps", "1", "--warmup", "0", "--cpu-seconds", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "logL evals/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_every_workload_builds(name):
    wl, spec = bench.make_workload(name)
    text = bench.workload_description(wl, spec)
    assert wl.name in text and spec["text"] in text
    if spec.get("tmarg_nodes"):
        params = bench.tmarg_params(wl)
        tc = params[bench.si.IDX["tc"]]
        assert tc.mode == bench.si.MODE_MARG and tc.kind == bench.si.PRIOR_UNIFORM
        assert (tc.lo, tc.hi) == (wl.params[bench.si.IDX["tc"]].lo, wl.params[bench.si.IDX["tc"]].hi)
