"""The oracle's pins must catch plausible mistakes. Each case plants one
mistake in a copy of oracle/dd_oracle.c: a dropped term, a wrong sign, scale,
index or rounding, a transposed operand, a missing channel. It builds that
copy and runs tests/test_oracle_pins.py against it in a subprocess, and some
pin must fail. The unchanged copy must pass every pin, so a failure comes
from the planted mistake, not from the harness. The real oracle is never
modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, text in dd_oracle.c that occurs exactly once, replacement)
MUTANTS = [
    ("shift_sign", "(inv_f2 - inv_ref2)", "(inv_ref2 - inv_f2)"),
    ("shift_scale", "delay_s / t_samp_s", "delay_s * t_samp_s"),
    ("shift_truncates", "llround(samples)", "(long long)samples"),
    ("shift_dm_dropped", "(ORACLE_DISPERSION_K * dm[d])", "(ORACLE_DISPERSION_K)"),
    ("forward_weight_dropped",
     "double term = w[c] * in[((int64_t)b * n_chan + c) * stride + t + k];",
     "double term = in[((int64_t)b * n_chan + c) * stride + t + k];"),
    ("forward_shift_dropped",
     "double term = w[c] * in[((int64_t)b * n_chan + c) * stride + t + k];",
     "double term = w[c] * in[((int64_t)b * n_chan + c) * stride + t];"),
    ("forward_shift_transposed",
     "int64_t k = shift[(int64_t)d * n_chan + c];\n                    double term",
     "int64_t k = shift[(int64_t)c * n_dm + d];\n                    double term"),
    ("forward_last_channel_missing",
     "for (int c = 0; c < n_chan; ++c) {\n                    int64_t k = shift[(int64_t)d * n_chan + c];\n"
     "                    double term",
     "for (int c = 0; c + 1 < n_chan; ++c) {\n                    int64_t k = shift[(int64_t)d * n_chan + c];\n"
     "                    double term"),
    ("forward_u8_weight_dropped",
     "acc += wq[c] * (int64_t)in[((int64_t)b * n_chan + c) * stride + t + k];",
     "acc += (int64_t)in[((int64_t)b * n_chan + c) * stride + t + k];"),
    ("points_weight_dropped", "double term = w[c] * row0[", "double term = row0["),
    ("points_u8_shift_dropped",
     "acc += wq[c] * (int64_t)row0[(int64_t)c * stride + pt[i] + k];",
     "acc += wq[c] * (int64_t)row0[(int64_t)c * stride + pt[i]];"),
    ("adjoint_shift_dropped",
     "gin[((int64_t)b * n_chan + c) * stride + t + k] += w[c] * gv;",
     "gin[((int64_t)b * n_chan + c) * stride + t] += w[c] * gv;"),
    ("adjoint_weight_dropped", "+ t + k] += w[c] * gv;", "+ t + k] += gv;"),
    ("grad_w_scale", "for (int64_t t = 0; t < n_out; ++t) acc += grow[t] * irow[t];",
     "for (int64_t t = 0; t < n_out; ++t) acc += 2.0 * grow[t] * irow[t];"),
    ("adjoint_points_weight_dropped", "double term = w[pc[i]] * g[", "double term = g["),
    ("grad_w_channels_input_dropped", "double term = grow[t] * irow[t];",
     "double term = grow[t];"),
]


def _run_pins_on(tmp_path, source):
    """Builds `source` as the oracle in tmp_path and runs the pins against
    it; returns the pytest subprocess result."""
    dst = tmp_path / "oracle"
    shutil.copytree(ORACLE_DIR, dst, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    (dst / "dd_oracle.c").write_text(source)
    runner = ("import sys; sys.path.insert(0, %r); import oracle; "
              "assert oracle.__file__.startswith(%r), oracle.__file__; "
              "import pytest; sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', %r]))"
              % (str(tmp_path), str(tmp_path), PINS))
    return subprocess.run([sys.executable, "-c", runner], cwd=ROOT, capture_output=True,
                          text=True, timeout=600)


def test_unchanged_copy_passes_every_pin(tmp_path):
    src = open(os.path.join(ORACLE_DIR, "dd_oracle.c")).read()
    r = _run_pins_on(tmp_path, src)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name,orig,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, repl):
    src = open(os.path.join(ORACLE_DIR, "dd_oracle.c")).read()
    assert src.count(orig) == 1, "mutation site of %s is not unique" % name
    r = _run_pins_on(tmp_path, src.replace(orig, repl))
    # a pin failed (pytest exit 1), rather than an import or build error
    assert r.returncode == 1 and " failed" in r.stdout, (
        "planted mistake %s was not caught:\n%s%s" % (name, r.stdout[-2000:], r.stderr[-1000:]))
