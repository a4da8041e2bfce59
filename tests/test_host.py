"""Host-side checks of libdd.so that need no GPU: the library loads, exports
every function include/dd.h declares, its Eq. 1 delay table equals the
oracle's exactly, and argument errors come back as status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
from paper_1601_05052_gb300 import _lib, compute_shifts, DDError, variants

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(dd_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    lib = _lib.load()
    names = _declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == {s[0] for s in _lib.SIGNATURES}
    assert lib.dd_version() == 1
    assert lib.dd_status_str(0) == b"DD_OK" and lib.dd_status_str(5) == b"DD_ERR_TIMEOUT"


@pytest.mark.parametrize("name", ["lband64", "apertif_survey", "lowfreq256_u8", "diff16_512ch", "lofar"])
def test_shift_table_equals_oracle_exactly(name):
    s = synth.setup(name)
    ref = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    got = compute_shifts(s.freqs(), s.f_ref, s.t_samp, s.dms())
    assert got.dtype == np.int32
    np.testing.assert_array_equal(got, ref)


def test_shift_table_any_order_and_random_setups():
    rng = np.random.default_rng(17)
    for _ in range(20):
        C, D = int(rng.integers(1, 300)), int(rng.integers(1, 300))
        f = rng.uniform(100.0, 2000.0, C)
        fr = f.max() * rng.uniform(1.0, 1.2)
        dm = rng.uniform(0.0, 500.0, D)
        ts = rng.uniform(1e-6, 1e-3)
        ref = oracle.shift_table(f, fr, ts, dm)
        if ref.max() > 2 ** 30:
            continue
        np.testing.assert_array_equal(compute_shifts(f, fr, ts, dm), ref)


def test_shift_table_errors():
    with pytest.raises(DDError) as e:
        compute_shifts([1500.0, 1400.0], 1400.0, 1e-4, [10.0])
    assert e.value.status == 1
    with pytest.raises(DDError):
        compute_shifts([1400.0], 1400.0, 0.0, [1.0])
    with pytest.raises(DDError):
        compute_shifts([1400.0], 1400.0, 1e-4, [float("nan")])
    with pytest.raises(DDError):
        compute_shifts([1.0, 2.0], 2.0, 1e-12, [1e6])  # beyond 2^30 samples


def test_plan_argument_errors_are_reported_before_any_device_call():
    lib = _lib.load()
    h = ctypes.c_void_p()
    f = np.array([1400.0, 1500.0])
    dm = np.array([0.0, 1.0])
    # n_out < 1
    st = lib.dd_plan_create(ctypes.byref(h), 2, f.ctypes.data, 1500.0, 1e-4, 2, dm.ctypes.data,
                            0, 1, 0)
    assert st == 1 and not h.value
    # bad dtype
    st = lib.dd_plan_create(ctypes.byref(h), 2, f.ctypes.data, 1500.0, 1e-4, 2, dm.ctypes.data,
                            16, 1, 9)
    assert st == 1
    # negative shift in an explicit table
    sh = np.array([[0, -1]], np.int32)
    st = lib.dd_plan_create_from_shifts(ctypes.byref(h), 2, 1, sh.ctypes.data, 8, 1, 0)
    assert st == 1 and b"shifts" in lib.dd_last_error_message()
    assert lib.dd_get_last_error() == 1
    # null plan handles
    assert lib.dd_execute(None, None, None, None, None) == 1
    assert lib.dd_adjoint(None, None, None, None, None, None, None) == 1
    assert lib.dd_plan_input_len(None) == -1


def test_variant_grid():
    vs = variants()
    assert len(vs) == _lib.load().dd_variant_count() and len(vs) > 50
    keys = {(v["kind"], v["dm_per_thread"], v["samples_per_thread"]) for v in vs}
    assert (0, 4, 4) in keys and (1, 8, 9) in keys and (2, 4, 8) in keys and (4, 8, 4) in keys
    for v in vs:
        assert v["warps_dm"] * v["warps_time"] <= (16 if v["kind"] in (4, 6) else 8)
        assert v["kind"] in (0, 1, 2, 3, 4, 5, 6) and (v["kind"] != 1 or v["samples_per_thread"] % 2 == 1)
        assert v["chans_per_stage"] in (4, 8, 16, 32) and 2 <= v["stages"] <= 4
    # kind 4 covers DM tiles of 128 trials
    assert any(v["kind"] == 4 and v["dm_per_thread"] * v["warps_dm"] == 128 for v in vs)


def test_plan_statistics_on_a_hand_table():
    """The plan statistics tool counts relative delay patterns per (DM tile,
    channel group) and equal adjacent delays on a table worked by hand."""
    from paper_1601_05052_gb300 import plan_stats
    sh = np.array([[0, 0, 0, 0],
                   [3, 2, 1, 0],
                   [6, 4, 2, 0],
                   [4, 3, 2, 1]])  # row 3 = row 1's pattern, base delay 1
    count, span = plan_stats.delay_patterns(sh, dt=4, group=4)
    assert count.tolist() == [[3]] and span.tolist() == [[1]]
    count, span = plan_stats.delay_patterns(sh, dt=2, group=2)
    # tile 0: groups (c0,c1): rel (0,0),(1,0) -> 2; (c2,c3): (0,0),(1,0) -> 2
    # tile 1: (c0,c1): (2,0),(1,0) -> 2; (c2,c3): (2,0),(1,0) -> 2
    assert count.tolist() == [[2, 2], [2, 2]]
    assert plan_stats.shared_adjacent_delays(np.array([[0, 1], [0, 2]])) == 0.5
    lane, sub, ratio = plan_stats.shared_words(sh, dt=4, ts=8, group=4)
    assert lane == 4 * 8 * 4
    assert sub == 4 * 8 * 1 + (1 + 3 * 8) * 5 and ratio == lane / sub
