"""GPU parity of the forward kernel against the FP64 oracle: every input type,
ragged shapes spanning several tiles, edge cases, the variant grid, and the
full-size survey workload at the benchmark's launch configuration (sampled)."""
import zlib

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1601_05052_gb300 import Plan, variants
from gpu_util import (assert_float_parity, check_full, points_by_beam, random_case, to_dev,
                      weights_dev)

pytestmark = pytest.mark.gpu
DTYPES = ["f32", "f16", "bf16", "u8"]


def _setup_case(name, dtype, wkind, seed):
    s = synth.setup(name).with_(dtype=dtype)
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    pulses = synth.pulse_plan(s, seed, fixed=(40, 1000, 5.0))
    x = synth.make_input(s, sh, seed=seed, pulses=pulses)
    w = synth.make_weights(s.n_chan, seed, wkind)
    if dtype == "u8":
        w = synth.quantize_weights_q8(w)
    return s, sh, x, w


def test_64ch_64dm_4096_plain_f32_full():
    """64 channels, 64 trials, 4096 samples, FP32, unit weights, one pulse."""
    s, sh, x, w = _setup_case("lband64", "f32", "ones", 1)
    plan = Plan.from_setup(s)
    np.testing.assert_array_equal(plan.shifts(), sh)
    out = check_full(plan, x, w, sh, "f32", "lband64")
    d, t = np.unravel_index(np.argmax(out[0]), out[0].shape)
    assert t == 1000 and abs(int(d) - 40) <= 1
    plan.check_device()


@pytest.mark.parametrize("dtype", ["u8", "f16", "bf16"])
def test_64ch_64dm_4096_precision_forms_full(dtype):
    """Workload 1's shapes and pulse with weights U(0.5,1.5), 5% masked:
    u8 bit-exact (int32), f16/bf16 within 1e-4 * sum|w*in|."""
    s, sh, x, w = _setup_case("lband64_" + dtype, dtype, "uniform", 3)
    plan = Plan.from_setup(s)
    check_full(plan, x, w, sh, dtype, "lband64 " + dtype)
    plan.check_device()


RAGGED = [  # (B, C, D, S, max_shift)
    (3, 37, 29, 1000, 150),
    (2, 5, 70, 333, 900),
    (1, 130, 3, 2049, 20),
    (1, 1, 1, 1, 0),
    (2, 64, 33, 4097, 4000),
]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("case", RAGGED)
def test_ragged_shapes_default_variant(dtype, case):
    rng = np.random.default_rng(zlib.crc32(repr((dtype, case)).encode()))
    sh, x, w = random_case(rng, *case, dtype=dtype)
    plan = Plan(shifts=sh, n_out=case[3], batch=case[0], dtype=dtype)
    check_full(plan, x, w, sh, dtype, "ragged %s %s" % (dtype, case))


@pytest.mark.parametrize("dtype", DTYPES)
def test_non_monotone_tables_and_dm0(dtype):
    rng = np.random.default_rng(5)
    sh, x, w = random_case(rng, 2, 19, 23, 700, 300, dtype, monotone=False)
    plan = Plan(shifts=sh, n_out=700, batch=2, dtype=dtype)
    check_full(plan, x, w, sh, dtype, "non-monotone")
    # Section IV-C: all trials at DM 0 -> every row is the weighted channel sum
    sh0, x0, w0 = random_case(rng, 1, 50, 17, 900, 0, dtype)
    plan0 = Plan(shifts=sh0, n_out=900, batch=1, dtype=dtype)
    out = check_full(plan0, x0, w0, sh0, dtype, "dm0")
    assert (out[0] == out[0, :1]).all()


def _variant_subset():
    vs = variants()
    picked, seen = [], set()
    for v in vs:
        key = (v["kind"], v["dm_per_thread"], v["samples_per_thread"], v["warps_dm"],
               v["warps_time"])
        if key in seen:
            continue
        seen.add(key)
        picked.append(v)
    # also every staging depth / chunk size once
    for v in vs:
        if v["warps_dm"] == 4 and ((v["kind"], v["dm_per_thread"], v["samples_per_thread"])
                                   in ((0, 4, 4), (1, 8, 9), (2, 4, 8), (3, 8, 4))):
            picked.append(v)
    return picked


@pytest.mark.parametrize("dtype", DTYPES)
def test_every_variant_shape(dtype):
    rng = np.random.default_rng(77)
    sh, x, w = random_case(rng, 2, 41, 45, 1500, 260, dtype)
    plan = Plan(shifts=sh, n_out=1500, batch=2, dtype=dtype)
    xd, wd = to_dev(x, dtype), weights_dev(w, dtype)
    if dtype == "u8":
        ref = oracle.forward_u8(x, w, sh, 1500)
    else:
        ref, ab = oracle.forward(x, w, sh, 1500, dtype=dtype, with_absum=True)
    n = 0
    for v in _variant_subset():
        try:
            plan.variant = v
        except Exception:
            continue  # does not fit this plan
        out = plan.execute(xd, wd).cpu().numpy()
        if dtype == "u8":
            np.testing.assert_array_equal(out.astype(np.int64), ref, err_msg=str(v))
        else:
            assert_float_parity(out, ref, ab, what=str(v))
        n += 1
    assert n >= 50
    plan.check_device()


@pytest.mark.parametrize("dtype", DTYPES)
def test_subband_kinds_every_shape(dtype):
    """The sub-band kinds (2, 3, 4) need delay tables whose channel groups
    share few relative patterns per DM tile, as Eq. 1 tables do; random
    tables never fit them. Ragged everywhere: 102 channels (a last group of
    2), 300 trials, 1100 samples, 2 beams."""
    from paper_1601_05052_gb300 import compute_shifts
    C, D, S = 102, 300, 1100
    freqs = 1420.0 + np.arange(C) * (300.0 / 1024)
    sh = compute_shifts(freqs, freqs[-1], 50e-6, np.arange(D) * 0.25).astype(np.int64)
    rng = np.random.default_rng(78)
    t_in = S + int(sh.max())
    stride = synth.padded_stride(t_in, dtype)
    xf = rng.standard_normal((2, C, stride)).astype(np.float32)
    xf[:, :, t_in:] = np.nan
    w = rng.uniform(-0.5, 1.5, C).astype(np.float32)
    if dtype == "f32":
        x = xf
    elif dtype == "f16":
        x = xf.astype(np.float16)
    elif dtype == "bf16":
        x = synth.to_bf16_bits(xf)
    else:
        x = synth.quantize_u8(np.nan_to_num(xf, nan=7.0))
        w = synth.quantize_weights_q8(w)
    plan = Plan(shifts=sh, n_out=S, batch=2, dtype=dtype)
    xd, wd = to_dev(x, dtype), weights_dev(w, dtype)
    if dtype == "u8":
        ref = oracle.forward_u8(x, w, sh, S)
    else:
        ref, ab = oracle.forward(x, w, sh, S, dtype=dtype, with_absum=True)
    ran = {}
    for v in variants():
        if v["kind"] not in (2, 3, 4, 6) or v["stages"] == 4:
            continue
        try:
            plan.variant = v
        except Exception:
            continue  # too many patterns for this tile shape
        out = plan.execute(xd, wd).cpu().numpy()
        if dtype == "u8":
            np.testing.assert_array_equal(out.astype(np.int64), ref, err_msg=str(v))
        else:
            assert_float_parity(out, ref, ab, what=str(v))
        ran[v["kind"]] = ran.get(v["kind"], 0) + 1
    assert all(ran.get(k, 0) >= 3 for k in (2, 3, 4)) and ran.get(6, 0) >= 1, ran
    plan.check_device()


def test_subband_u8_wide_integer_weights():
    """8-bit sub-band kernels with integer weights far from the Q8 range:
    random 16-bit values, both ends of the 16-bit range, zeros, and weights
    beyond it (up to 2^20, negative too), with sums that still fit INT32;
    every sub-band kind must stay bit-exact."""
    from paper_1601_05052_gb300 import compute_shifts
    C, D, S = 102, 300, 1100
    freqs = 1420.0 + np.arange(C) * (300.0 / 1024)
    sh = compute_shifts(freqs, freqs[-1], 50e-6, np.arange(D) * 0.25).astype(np.int64)
    rng = np.random.default_rng(79)
    t_in = S + int(sh.max())
    stride = synth.padded_stride(t_in, "u8")
    x = rng.integers(0, 256, size=(2, C, stride)).astype(np.uint8)
    w = rng.integers(-32768, 32768, size=C).astype(np.int32)
    w[[0, 5, 10]] = [-32768, 32767, 0]
    w[[17, 42, 64, 101]] = [40000, -40000, 1 << 20, -32769]
    w[rng.random(C) < 0.05] = 0
    plan = Plan(shifts=sh, n_out=S, batch=2, dtype="u8")
    xd, wd = to_dev(x, "u8"), weights_dev(w, "u8")
    ref = oracle.forward_u8(x, w, sh, S)
    assert np.abs(ref).max() < 2**31
    ran = {}
    for v in variants():
        if v["kind"] not in (2, 3, 4, 6) or v["stages"] == 4:
            continue
        try:
            plan.variant = v
        except Exception:
            continue
        out = plan.execute(xd, wd).cpu().numpy()
        np.testing.assert_array_equal(out.astype(np.int64), ref, err_msg=str(v))
        ran[v["kind"]] = ran.get(v["kind"], 0) + 1
    assert all(ran.get(k, 0) >= 1 for k in (2, 3, 4, 6)), ran
    plan.check_device()


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_lane_strided_shared_delays(dtype):
    """Kind 5 loads a channel's operands once for adjacent trials that share
    its delay. An Eq. 1 table at low DMs (64 channels over 1400-1500 MHz,
    DM step 0.5, 64 us) has many such pairs, mixed with channels that have
    none; every CTA shape of kinds 0 and 5 must match the oracle."""
    from paper_1601_05052_gb300 import compute_shifts
    C, D, S = 64, 40, 777
    freqs = 1400.0 + np.arange(C) * (100.0 / C)
    sh = compute_shifts(freqs, freqs[-1], 64e-6, np.arange(D) * 0.5).astype(np.int64)
    assert (sh[1:] == sh[:-1]).mean() > 0.2 and (sh[1:] != sh[:-1]).any()
    rng = np.random.default_rng(79)
    t_in = S + int(sh.max())
    stride = synth.padded_stride(t_in, dtype)
    xf = rng.standard_normal((2, C, stride)).astype(np.float32)
    xf[:, :, t_in:] = np.nan
    w = rng.uniform(-0.5, 1.5, C).astype(np.float32)
    x = {"f32": xf, "f16": xf.astype(np.float16), "bf16": synth.to_bf16_bits(xf)}[dtype]
    plan = Plan(shifts=sh, n_out=S, batch=2, dtype=dtype)
    xd, wd = to_dev(x, dtype), weights_dev(w, dtype)
    ref, ab = oracle.forward(x, w, sh, S, dtype=dtype, with_absum=True)
    n = {0: 0, 5: 0}
    for v in variants():
        if v["kind"] not in n or v["stages"] == 4:
            continue
        try:
            plan.variant = v
        except Exception:
            continue
        assert_float_parity(plan.execute(xd, wd).cpu().numpy(), ref, ab, what=str(v))
        n[v["kind"]] += 1
    assert n[0] >= 20 and n[5] >= 6, n
    plan.check_device()


def test_execute_host_matches_device_path():
    rng = np.random.default_rng(9)
    sh, x, w = random_case(rng, 2, 30, 40, 800, 100, "f32")
    plan = Plan(shifts=sh, n_out=800, batch=2)
    dev = plan.execute(to_dev(x, "f32"), weights_dev(w, "f32")).cpu()
    hx = torch.from_numpy(x).pin_memory()
    hw = torch.from_numpy(w).pin_memory()
    hout = torch.empty(plan.out_shape, dtype=torch.float32).pin_memory()
    plan.execute_host(hx, hw, hout)  # pinned: pulled and written over the CPU-GPU link
    assert torch.equal(dev, hout)
    px = torch.from_numpy(x.copy())  # pageable: staged through device mirrors
    pout = torch.zeros(plan.out_shape, dtype=torch.float32)
    plan.execute_host(px, torch.from_numpy(w.copy()), pout)
    assert torch.equal(dev, pout)
    for _ in range(2):  # repeated calls reuse the mirrors
        hout.zero_()
        plan.execute_host(hx, hw, hout)
        assert torch.equal(dev, hout)


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_execute_host_segmented_pipeline(dtype):
    """Pinned input with many time tiles: the input is pulled in segments (an
    SM copy for the first, the copy engine for the rest) and each segment's
    forward starts once its columns are in; results equal the device path.
    Also a sub-band variant (Eq. 1 table) and a repeated call."""
    from paper_1601_05052_gb300 import compute_shifts
    rng = np.random.default_rng(12)
    sh, x, w = random_case(rng, 2, 36, 40, 9000, 700, dtype)
    plan = Plan(shifts=sh, n_out=9000, batch=2, dtype=dtype)
    freqs = 1420.0 + np.arange(64) * (300.0 / 1024)
    sh2 = compute_shifts(freqs, freqs[-1], 50e-6, np.arange(128) * 0.25).astype(np.int64)
    plan2 = Plan(shifts=sh2, n_out=7000, batch=1, dtype=dtype)
    t_in2 = 7000 + int(sh2.max())
    x2 = rng.integers(0, 255, (1, 64, synth.padded_stride(t_in2, dtype))).astype(
        np.uint8 if dtype == "u8" else np.float32)
    w2 = w[:1].repeat(64) if dtype == "u8" else rng.uniform(0.5, 1.5, 64).astype(np.float32)
    for pl, xx, ww in ((plan, x, w), (plan2, x2, w2)):
        dev = pl.execute(to_dev(xx, dtype), weights_dev(ww, dtype)).cpu()
        hx = torch.from_numpy(np.ascontiguousarray(xx)).pin_memory()
        hw = torch.from_numpy(np.ascontiguousarray(ww)).pin_memory()
        hout = torch.empty(pl.out_shape, dtype=dev.dtype).pin_memory()
        for _ in range(2):
            hout.zero_()
            pl.execute_host(hx, hw, hout)
            assert torch.equal(dev, hout), pl.variant
    assert plan2.variant["kind"] in (2, 4, 6)


def test_kernel_shared_memory_limit_is_only_raised():
    """Variants of one compiled kernel differ in dynamic shared memory (here
    16 against 32 channels per stage). A call that needs less than an
    earlier launch (the end-to-end pipeline's occupancy query, or another
    plan's launch) must leave the kernel's limit high enough for that
    earlier plan's next launch."""
    from paper_1601_05052_gb300 import compute_shifts
    freqs = 1420.0 + np.arange(256) * (300.0 / 1024)
    sh = compute_shifts(freqs, freqs[-1], 50e-6, np.arange(256) * 0.25).astype(np.int64)
    V = dict(kind=6, dm_per_thread=4, samples_per_thread=8, warps_dm=16, warps_time=1,
             stages=2)
    big = Plan(shifts=sh, n_out=2000)
    big.variant = dict(V, chans_per_stage=32)
    small = Plan(shifts=sh, n_out=2000)
    small.variant = dict(V, chans_per_stage=16)
    rng = np.random.default_rng(31)
    x = rng.standard_normal(big.in_shape).astype(np.float32)
    w = np.ones(256, np.float32)
    xd, wd = to_dev(x, "f32"), weights_dev(w, "f32")
    first = big.execute(xd, wd).cpu()
    hx, hw = torch.from_numpy(x).pin_memory(), torch.from_numpy(w).pin_memory()
    hout = torch.empty(small.out_shape).pin_memory()
    small.execute_host(hx, hw, hout)
    small.execute(xd, wd)
    assert torch.equal(big.execute(xd, wd).cpu(), first)
    ref, ab = oracle.forward(x, w, sh, 2000, with_absum=True)
    assert_float_parity(first.numpy(), ref, ab, what="32 channels per stage")
    assert_float_parity(hout.numpy(), ref, ab, what="16 channels per stage, end to end")
    big.check_device()


def test_tuned_variant_stays_correct():
    rng = np.random.default_rng(10)
    sh, x, w = random_case(rng, 1, 96, 64, 3000, 400, "f32")
    plan = Plan(shifts=sh, n_out=3000, batch=1)
    rep = plan.tune(budget_ms=3000)
    assert rep["n_tried"] >= 2 and rep["best_gflops"] >= rep["mean_gflops"]
    assert plan.variant == rep["best"]
    check_full(plan, x, w, sh, "f32", "tuned")


def test_tuning_cache_restores_the_tuned_variant(tmp_path, monkeypatch):
    """dd_tune records its winner under DD_TUNE_CACHE; a new plan of the same
    problem starts from it, a plan of another problem does not."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("DD_TUNE_CACHE", str(cache))
    rng = np.random.default_rng(11)
    sh, x, w = random_case(rng, 1, 64, 48, 2000, 300, "f32")
    plan = Plan(shifts=sh, n_out=2000, batch=1)
    default = plan.variant
    rep = plan.tune(budget_ms=2000)
    assert cache.read_text().count("\n") == 1
    # force a non-default winner into the cache so that the restore is visible
    other = next(v for v in variants() if v["kind"] == 0 and v != default
                 and _fits(sh, 2000, v))
    line = cache.read_text().split()[0]
    cache.write_text(cache.read_text() + "%s %d %d %d %d %d %d %d\n" % (
        line, other["kind"], other["dm_per_thread"], other["samples_per_thread"],
        other["warps_dm"], other["warps_time"], other["chans_per_stage"], other["stages"]))
    again = Plan(shifts=sh, n_out=2000, batch=1)
    assert again.variant == other
    check_full(again, x, w, sh, "f32", "cached")
    sh2 = sh.copy()
    sh2[0, 0] += 1
    assert Plan(shifts=sh2, n_out=2000, batch=1).variant == default
    assert rep["best"] == plan.variant
    monkeypatch.delenv("DD_TUNE_CACHE")
    assert Plan(shifts=sh, n_out=2000, batch=1).variant == default


def _fits(sh, n_out, v):
    p = Plan(shifts=sh, n_out=n_out, batch=1)
    try:
        p.variant = v
        return True
    except Exception:
        return False


def test_survey_scale_f32_sampled():
    """The benchmark workload (1024 ch, 2048 trials, 20000 samples, FP32) in
    the launch configuration the benchmark times: sampled outputs, plus the
    ten injected pulses."""
    s = synth.setup("apertif_survey")
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    pulses = synth.pulse_plan(s, 2, n_per_beam=10)
    x = synth.make_input(s, sh, seed=2, pulses=pulses)
    w = synth.make_weights(s.n_chan, 2, "ones")
    plan = Plan.from_setup(s)
    out = plan.execute(to_dev(x, "f32"), weights_dev(w, "f32"))
    torch.cuda.synchronize()
    rng = np.random.default_rng(22)
    n = 4000
    pd = np.concatenate([rng.integers(0, s.n_dm, n), [p[1] for p in pulses],
                         [0, s.n_dm - 1, s.n_dm - 1, 0]])
    pt = np.concatenate([rng.integers(0, s.n_out, n), [p[2] for p in pulses],
                         [0, s.n_out - 1, 0, s.n_out - 1]])
    pb = np.zeros_like(pd)
    ref, ab = oracle.forward_points(x, w, sh, pb, pd, pt)
    got = out[0][torch.from_numpy(pd).cuda(), torch.from_numpy(pt).cuda()].cpu().numpy()
    assert_float_parity(got, ref, ab, what="apertif_survey sampled")
    # each pulse is recovered at its own trial and time
    for (_, d, t0, a) in pulses:
        col = out[0, :, t0].cpu().numpy()
        assert col[d] > 0.5 * a * s.n_chan
    # the end-to-end path the benchmark's e2e times (pinned host buffers,
    # segmented pulls and launches) gives the device path's array exactly
    hx = torch.from_numpy(x).pin_memory()
    hw = torch.from_numpy(w).pin_memory()
    hout = torch.empty(plan.out_shape, dtype=torch.float32).pin_memory()
    plan.execute_host(hx, hw, hout)
    assert torch.equal(hout, out.cpu())
    plan.check_device()


@pytest.mark.parametrize("dtype,wkind", [("u8", "uniform"), ("u8", "ones"), ("f16", "uniform"),
                                         ("bf16", "uniform")])
def test_survey_scale_narrow_inputs_sampled(dtype, wkind):
    """The survey workload (1024 ch, 2048 trials, 20000 samples) with 8-bit
    and 16-bit input in the plan's default variant (the wide sub-band kind
    the benchmark times for these types), weights U(0.5, 1.5) with 5 %
    masked (Q8 integers for 8-bit input), or unit weights (Q8: 256 for every
    channel, as the benchmark times 8-bit input): 4000 sampled outputs, the
    ten pulses and the corners, bit-exact for u8, within 1e-4 * sum|w*in| for
    f16 / bf16."""
    s = synth.setup("apertif_survey").with_(dtype=dtype)
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    pulses = synth.pulse_plan(s, 2, n_per_beam=10)
    x = synth.make_input(s, sh, seed=2, pulses=pulses)
    w = synth.make_weights(s.n_chan, 2, wkind)
    if dtype == "u8":
        w = synth.quantize_weights_q8(w)
    plan = Plan.from_setup(s)
    assert plan.variant["kind"] == 4, plan.variant
    out = plan.execute(to_dev(x, dtype), weights_dev(w, dtype))
    torch.cuda.synchronize()
    rng = np.random.default_rng(23)
    n = 4000
    pd = np.concatenate([rng.integers(0, s.n_dm, n), [p[1] for p in pulses],
                         [0, s.n_dm - 1, s.n_dm - 1, 0]])
    pt = np.concatenate([rng.integers(0, s.n_out, n), [p[2] for p in pulses],
                         [0, s.n_out - 1, 0, s.n_out - 1]])
    pb = np.zeros_like(pd)
    got = out[0][torch.from_numpy(pd).cuda(), torch.from_numpy(pt).cuda()].cpu().numpy()
    ref, ab = points_by_beam(x, w, sh, pb, pd, pt, dtype)
    if dtype == "u8":
        np.testing.assert_array_equal(got.astype(np.int64), ref)
    else:
        assert_float_parity(got, ref, ab, what="apertif_survey %s sampled" % dtype)
    plan.check_device()


def test_bounded_wait_reports_timeout_and_context_survives():
    """A kernel waiting on a barrier nothing completes gives up after its
    budget, the host reads DD_ERR_TIMEOUT, and the next launch still works."""
    import ctypes
    from paper_1601_05052_gb300 import DDError, _lib
    rng = np.random.default_rng(12)
    sh, x, w = random_case(rng, 1, 8, 8, 300, 20, "f32")
    plan = Plan(shifts=sh, n_out=300, batch=1)
    plan.check_device()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(_lib.load().dd_debug_wait_timeout(plan._h, 50000, st))  # 50 ms budget
    with pytest.raises(DDError) as e:
        plan.check_device()
    assert e.value.status == 5  # DD_ERR_TIMEOUT
    plan.check_device()  # the error word was cleared
    check_full(plan, x, w, sh, "f32", "after timeout")


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_stream_equals_one_long_dedispersion(dtype):
    """Pushing K chunks through a stream gives the dedispersion of the whole
    concatenated input with M leading zeros, output delayed by M samples."""
    from paper_1601_05052_gb300 import Stream
    rng = np.random.default_rng(31)
    C, D, S, K, M = 13, 11, 160, 5, 400
    sh = np.sort(rng.integers(0, M + 1, size=(D, C)), axis=0)
    sh[-1, 0] = M
    plan = Plan(shifts=sh, n_out=S, batch=2, dtype=dtype)
    st = Stream(plan)
    assert st.latency == M
    xf = rng.standard_normal((2, C, K * S)).astype(np.float32)
    x = xf if dtype == "f32" else synth.quantize_u8(xf)
    w = rng.uniform(0.5, 1.5, C).astype(np.float32)
    if dtype == "u8":
        w = synth.quantize_weights_q8(w)
    wd = weights_dev(w, dtype)
    outs = [st.push(to_dev(np.ascontiguousarray(x[:, :, k * S:(k + 1) * S]), dtype), wd).cpu().numpy()
            for k in range(K)]
    got = np.concatenate(outs, axis=2)
    full = np.zeros((2, C, M + K * S + 16), dtype=x.dtype)
    full[:, :, M:M + K * S] = x
    if dtype == "u8":
        ref = oracle.forward_u8(full, w, sh, K * S)
        np.testing.assert_array_equal(got.astype(np.int64), ref)
    else:
        ref, ab = oracle.forward(full, w, sh, K * S, with_absum=True)
        assert_float_parity(got, ref, ab, what="stream")
    st.reset()
    again = st.push(to_dev(np.ascontiguousarray(x[:, :, :S]), dtype), wd).cpu().numpy()
    np.testing.assert_array_equal(again, outs[0])


def test_binding_rejects_buffers_the_kernels_cannot_take():
    """A caller's buffer pointer goes to a kernel as is: host tensors, other
    shapes or types, and non-contiguous views are refused before any launch."""
    from paper_1601_05052_gb300 import Batch
    rng = np.random.default_rng(41)
    sh, x, w = random_case(rng, 2, 9, 7, 100, 30, "f32")
    plan = Plan(shifts=sh, n_out=100, batch=2)
    xd, wd = to_dev(np.nan_to_num(x), "f32"), weights_dev(w, "f32")
    bad_outs = [torch.empty(plan.out_shape),  # host memory
                torch.empty((2, 7, 99), device="cuda"),  # shape
                torch.empty(plan.out_shape, dtype=torch.float16, device="cuda"),  # type
                torch.empty((2, 7, 200), device="cuda")[:, :, ::2]]  # non-contiguous
    for o in bad_outs:
        with pytest.raises(ValueError):
            plan.execute(xd, wd, out=o)
    with pytest.raises(ValueError):
        plan.execute(xd.cpu(), wd)
    g = torch.zeros(plan.out_shape, device="cuda")
    with pytest.raises(ValueError):
        plan.adjoint(g, wd, xd.half())  # grad_w needs the FP32 input
    with pytest.raises(ValueError):
        plan.adjoint(g, None, xd)  # grad_in needs the weights
    batch = Batch([plan])
    with pytest.raises(ValueError):
        batch.execute([xd, xd], [wd])
    with pytest.raises(ValueError):
        batch.execute([xd], [wd], [bad_outs[3]])
    # the end-to-end call reads and writes whole buffers of the plan's shapes
    hx, hw = torch.from_numpy(np.nan_to_num(x)), torch.from_numpy(w)
    hout = torch.empty(plan.out_shape)
    for args in ((hx[:1], hw, hout), (hx, hw[:-1], hout), (hx, hw, hout[:, :-1]),
                 (hx.half(), hw, hout), (hx, hw, hout.int()), (hx.cuda(), hw, hout)):
        with pytest.raises(ValueError):
            plan.execute_host(*args)
    ok = plan.execute(xd, wd, out=torch.empty(plan.out_shape, device="cuda"))
    ref, ab = oracle.forward(np.nan_to_num(x), w, sh, 100, with_absum=True)
    assert_float_parity(ok.cpu().numpy(), ref, ab, what="after refusals")


def test_set_variant_waits_for_this_plans_launches_only():
    """dd_plan_set_variant replaces the tables that launches read. It waits
    for the plan's own launches (on every stream they went to, more streams
    than it keeps slots for) instead of the whole device; each launch made
    before the change still reads the old, intact tables."""
    from paper_1601_05052_gb300 import compute_shifts
    C, D, S = 256, 512, 6000
    freqs = 1420.0 + np.arange(C) * (300.0 / C)
    sh = compute_shifts(freqs, freqs[-1], 50e-6, np.arange(D) * 0.25).astype(np.int64)
    rng = np.random.default_rng(42)
    plan = Plan(shifts=sh, n_out=S, batch=1)
    x = rng.standard_normal(plan.in_shape).astype(np.float32)
    w = rng.uniform(0.5, 1.5, C).astype(np.float32)
    xd, wd = to_dev(x, "f32"), weights_dev(w, "f32")
    kinds = [v for v in variants() if v["kind"] in (0, 4) and v["stages"] == 2
             and v["chans_per_stage"] == 16 and _fits(sh, S, v)][:3]
    assert len(kinds) >= 2
    streams = [torch.cuda.Stream() for _ in range(10)]
    outs = []
    for k, v in enumerate(kinds):
        plan.variant = v
        for st in streams:  # launches on 10 streams, then the next change at once
            o = torch.empty(plan.out_shape, device="cuda")
            with torch.cuda.stream(st):
                plan.execute(xd, wd, out=o, stream=st)
            outs.append(o)
    torch.cuda.synchronize()
    ref, ab = oracle.forward(x, w, sh, S, with_absum=True)
    for o in outs:
        assert_float_parity(o.cpu().numpy(), ref, ab, what="launch before a variant change")
    plan.check_device()



@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_launch_orders_give_identical_results(dtype):
    """The tiles' launch order (DM tiles fastest or time tiles fastest) only
    changes which CTAs run together: for every kernel kind the two orders give
    bit-identical outputs, equal to the oracle's, including on a segmented
    host pipeline launch."""
    from paper_1601_05052_gb300 import compute_shifts
    C, D, S, B = 70, 150, 3100, 2
    freqs = 1420.0 + np.arange(C) * (300.0 / C)
    sh = compute_shifts(freqs, freqs[-1], 50e-6, np.arange(D) * 0.25).astype(np.int64)
    rng = np.random.default_rng(43)
    plan = Plan(shifts=sh, n_out=S, batch=B, dtype=dtype)
    xf = rng.standard_normal(plan.in_shape).astype(np.float32)
    w = rng.uniform(0.5, 1.5, C).astype(np.float32)
    x = xf
    if dtype == "u8":
        x, w = synth.quantize_u8(xf), synth.quantize_weights_q8(w)
    xd, wd = to_dev(x, dtype), weights_dev(w, dtype)
    if dtype == "u8":
        ref = oracle.forward_u8(x, w, sh, S)
    else:
        ref, ab = oracle.forward(x, w, sh, S, with_absum=True)
    ran = 0
    for kind in (0, 1, 2, 3, 4, 5):
        cand = [v for v in variants() if v["kind"] == kind and v["stages"] == 2]
        for v in cand:
            try:
                plan.variant = v
            except Exception:
                continue
            assert plan.launch_order == "dm"
            first = plan.execute(xd, wd)
            plan.launch_order = "time"
            second = plan.execute(xd, wd)
            assert torch.equal(first, second), v
            if dtype == "u8":
                np.testing.assert_array_equal(second.cpu().numpy().astype(np.int64), ref)
            else:
                assert_float_parity(second.cpu().numpy(), ref, ab, what=str(v))
            hx = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
            hw = torch.from_numpy(np.ascontiguousarray(w)).pin_memory()
            hout = torch.empty(plan.out_shape, dtype=first.dtype).pin_memory()
            plan.execute_host(hx, hw, hout)
            assert torch.equal(first.cpu(), hout), v
            ran += 1
            break
    assert ran >= 5, ran
    from paper_1601_05052_gb300 import _lib
    assert _lib.load().dd_plan_set_launch_order(plan._h, 2) == 1  # DD_ERR_ARG
    assert plan.launch_order == "time"
    plan.check_device()


@pytest.mark.parametrize("dtype", ["f32", "u8", "f16", "bf16"])
def test_64ch_64dm_4096_tuned_full(dtype):
    """The 64-channel workload and its 8/16-bit forms in the variant the
    tuner picks for them (the benchmark replays that variant's launches from
    a CUDA graph): the whole output against the oracle, before and after
    tuning, also from inside a captured graph."""
    name = "lband64" if dtype == "f32" else "lband64_" + dtype
    s, sh, x, w = _setup_case(name, dtype, "ones" if dtype == "f32" else "uniform", 3)
    plan = Plan.from_setup(s)
    check_full(plan, x, w, sh, dtype, "default " + dtype)
    plan.tune(budget_ms=2000)
    check_full(plan, x, w, sh, dtype, "tuned %s %s" % (dtype, plan.variant))
    xd, wd = to_dev(x, dtype), weights_dev(w, dtype)
    out = torch.empty(plan.out_shape, dtype=plan.out_dtype, device="cuda")
    plan.execute(xd, wd, out)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(3):
            plan.execute(xd, wd, out)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    if dtype == "u8":
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64),
                                      oracle.forward_u8(x, w, sh, s.n_out))
    else:
        ref, ab = oracle.forward(x, w, sh, s.n_out, dtype=dtype, with_absum=True)
        assert_float_parity(out.cpu().numpy(), ref, ab, what="graph " + dtype)
    # a variant change after the capture keeps the captured tables alive
    plan.variant = dict(kind=0, dm_per_thread=4, samples_per_thread=4, warps_dm=4, warps_time=2,
                        chans_per_stage=8, stages=3)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    if dtype == "u8":
        np.testing.assert_array_equal(out.cpu().numpy().astype(np.int64),
                                      oracle.forward_u8(x, w, sh, s.n_out))
    plan.check_device()


@pytest.mark.parametrize("name,variant", [
    ("lband64_x96", dict(kind=5, dm_per_thread=4, samples_per_thread=8, warps_dm=8, warps_time=1,
                         chans_per_stage=16, stages=3)),
    ("lband64_4dm_x384", dict(kind=0, dm_per_thread=4, samples_per_thread=8, warps_dm=1,
                              warps_time=8, chans_per_stage=4, stages=3)),
])
def test_many_beam_points_sampled(name, variant):
    """The benchmark's 96-beam and HBM-bound 384-beam FP32 points (64
    channels over 1400-1500 MHz) in the variants it times: 4000 sampled
    outputs over all beams, plus the first and last beam's corners."""
    s = synth.setup(name)
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    x = synth.make_input(s, sh, seed=7, pulses=synth.pulse_plan(s, 7))
    w = synth.make_weights(s.n_chan, 7, "uniform")
    plan = Plan.from_setup(s)
    plan.variant = variant
    out = plan.execute(to_dev(x, "f32"), weights_dev(w, "f32"))
    torch.cuda.synchronize()
    rng = np.random.default_rng(25)
    n = 4000
    pb = np.concatenate([rng.integers(0, s.batch, n), [0, 0, s.batch - 1, s.batch - 1]])
    pd = np.concatenate([rng.integers(0, s.n_dm, n), [0, s.n_dm - 1, 0, s.n_dm - 1]])
    pt = np.concatenate([rng.integers(0, s.n_out, n), [0, s.n_out - 1, s.n_out - 1, 0]])
    got = out[torch.from_numpy(pb).cuda(), torch.from_numpy(pd).cuda(),
              torch.from_numpy(pt).cuda()].cpu().numpy()
    ref, ab = oracle.forward_points(x, w, sh, pb, pd, pt)
    assert_float_parity(got, ref, ab, what="%s %s" % (name, variant))
    plan.check_device()
