"""bench.py's JSON line keeps its contract: one line with the metric, the
whole-job value, the roofline of the forward kernel (with its ALU peak and the
HBM fraction beside it), the end-to-end number through dd_execute_host with
its host<->device bytes, the clocks sampled during the timed steps, the kernel
launch count and the real-time factor."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "4",
                        "--warmup", "3", "--no-extras", "--no-cpu-baseline"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["metric"] == d["unit"] == "DM-trial·samples/s"
    assert d["n_gpus"] == 1 and d["steps"] == 4 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    units = d["config"]["n_dm"] * d["config"]["n_out"] * d["config"]["beams_per_rank"]
    assert d["value"] == pytest.approx(units / (d["ms_per_step"] * 1e-3), rel=1e-9)
    roof = d["roofline"]
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"], rel=1e-9)
    assert 0 < roof["frac"] < 1.5
    assert 0 < roof["hbm"]["frac"] < 1.5
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] == 4
    assert d["dtype"] == "f32" and d["data"] == "synthetic"
    assert d["real_time"]["factor"] > 1
    assert "clocks" in d
