"""Host-side logic of the benchmark and the experiment report, on CPU: the
DRAM traffic recorded in the committed ncu summary is reported only for the
kernel sources and variant it was taken from, and the tuning-experiment table
is rendered from the run's own results."""
import json
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1601_05052_gb300 import experiments  # noqa: E402


def _profile_variant():
    text = open(os.path.join(ROOT, bench.TRAFFIC_PROFILE)).read()
    line = next(l for l in text.splitlines() if l.startswith("variant: "))
    return json.loads(line[len("variant: "):])


def test_recorded_traffic_matches_sources_and_variant():
    """The committed summary's figures are used only with the kernel sources
    and the variant they were taken from."""
    v = _profile_variant()
    text = open(os.path.join(ROOT, bench.TRAFFIC_PROFILE)).read()
    m = re.search(r"kernel source hash: ([0-9a-f]{16})", text)
    assert m
    current = text.replace(m.group(0), "kernel source hash: " + bench.kernel_hash())
    t = bench.recorded_traffic(v, current)
    assert t is not None and 1e8 < t < 3e8  # read + write bytes of one survey launch
    assert bench.recorded_traffic(dict(v, stages=v["stages"] + 1), current) is None
    stale = text.replace(m.group(0), "kernel source hash: 0123456789abcdef")
    assert bench.recorded_traffic(v, stale) is None
    # the committed file gives figures exactly when its hash is the sources' own
    assert (bench.recorded_traffic(v) is not None) == (m.group(1) == bench.kernel_hash())


def test_recorded_wavefronts_and_shared_memory_roofline():
    """The shared-memory figure follows the same gating as the traffic, and
    the roofline it gives is wavefronts x 128 bytes over the launch time
    against one wavefront per SM per clock."""
    v = _profile_variant()
    text = open(os.path.join(ROOT, bench.TRAFFIC_PROFILE)).read()
    m = re.search(r"kernel source hash: ([0-9a-f]{16})", text)
    current = text.replace(m.group(0), "kernel source hash: " + bench.kernel_hash())
    wf = bench.recorded_wavefronts(v, current)
    assert wf is not None and 1e8 < wf < 2e9
    assert bench.recorded_wavefronts(dict(v, kind=4), current) is None
    stale = text.replace(m.group(0), "kernel source hash: 0123456789abcdef")
    assert bench.recorded_wavefronts(v, stale) is None
    r = bench._smem_roofline(v, 2.0, 152, {"sm_max_mhz": 2000.0})
    if r["wavefronts"] is not None:
        assert abs(r["peak_gbs"] - 152 * 128 * 2.0) < 1e-6
        assert abs(r["frac"] - r["wavefronts"] * 128 / 2e-3 / 1e9 / r["peak_gbs"]) < 1e-12


def test_kernel_hash_is_stable_and_covers_the_sources():
    assert bench.kernel_hash() == bench.kernel_hash()
    assert len(bench.kernel_hash()) == 16
    for f in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, f)), f


def test_experiment_table_rendering():
    rows = lambda vals: [{"n_dm": n, "best_gflops": g, "mean_gflops": g / 2, "snr": 2.0,
                          "chebyshev": 0.25, "speedup_tuned_over_fixed": 1.1}
                         for n, g in vals]
    res = [{"setup": "apertif", "dm0_only": False, "instances": rows([(2, 100.0), (4, 210.4)])},
           {"setup": "apertif", "dm0_only": True, "instances": rows([(2, 120.0)])},
           {"setup": "lofar", "dm0_only": False, "instances": rows([(4, 50.0)])}]
    md = experiments.markdown(res).splitlines()
    assert md[0].startswith("| D | Apertif best GFLOP/s")
    assert md[2] == "| 2 | 100 | 50 | 2.00 | 0.25 | 1.10 | 120 | - | - |"
    assert md[3] == "| 4 | 210 | 105 | 2.00 | 0.25 | 1.10 | - | 50 | - |"
    assert len(md) == 4
