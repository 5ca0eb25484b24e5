"""The bench's JSON line on a GB300: one short run of `bench.py` (one timed
step of the 2e5-cell workload, the mixed path and its end-to-end leg) and
the keys, units and internal consistency of the line it prints."""
import json
import subprocess
import sys

import pytest

import bench

pytestmark = pytest.mark.gpu


def test_bench_line_contract():
    cmd = [sys.executable, "bench.py", "--steps", "1", "--warmup", "3", "--no-fp64", "--no-cpu", "--no-large",
           "--no-adjoint", "--no-hii", "--no-config5"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["data"] == "synthetic"
    cfg = d["config"]
    assert "workload" in cfg and cfg["n_sub"] == bench.N_SUB
    # value is the cell-updates of the timed step over its time
    assert d["value"] == pytest.approx(cfg["cells"] * cfg["n_sub"] / (d["ms_per_step"] * 1e-3), rel=1e-6)
    rf = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rf, k
    assert rf["bound"] in ("hbm", "alu", "tensor")
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"], rel=1e-2)
    assert 0 < rf["frac"] < 1.5
    sub = d["roofline_subcycle"]
    assert sub["bound"] == "hbm" and 0 < sub["frac"] < 1.5
    e2e = d["e2e"]
    assert e2e["unit"] == bench.UNIT and e2e["value"] > 0
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    # the end-to-end leg carries the copies, so it is no faster than the
    # device-resident step beyond timing noise
    assert e2e["value"] < 1.1 * d["value"]
    # five launches per subcycle (two chemistry passes, gradients, fluxes,
    # flux application), all of them the library's own kernels
    assert d["gpu_launches"] == 5 * bench.N_SUB * d["steps"]
    cl = d["clocks"]
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(cl)
