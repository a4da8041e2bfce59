"""GPU parity where neighbouring trials' delays differ by more than a time
tile, so each channel stages one window per run of touching trial windows
instead of their union: the paper's LOFAR setup with real DMs (Section IV:
32 channels of 0.195 MHz from 138 MHz, 5 us sampling, DM step 0.25, where
one DM step moves the lowest channel by ~900 samples) and a coarse DM grid
over a low band whose delay steps exceed 10^5 samples."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1601_05052_gb300 import DDError, Plan, variants
from gpu_util import assert_float_parity, points_by_beam, to_dev, weights_dev

pytestmark = pytest.mark.gpu


def _inputs(s, sh, dtype, seed, B=1):
    s = s.with_(dtype=dtype, batch=B)
    pulses = synth.pulse_plan(s, seed, amp=(4.0, 8.0))
    x = synth.make_input(s, sh, seed=seed, pulses=pulses)
    w = synth.make_weights(s.n_chan, seed, "uniform")
    if dtype == "u8":
        w = synth.quantize_weights_q8(w)
    return s, x, w


def _reference(x, w, sh, n_out, dtype):
    if dtype == "u8":
        return oracle.forward_u8(x, w, sh, n_out), None
    return oracle.forward(x, w, sh, n_out, dtype=dtype, with_absum=True)


def _check(out, ref, ab, dtype, what):
    if dtype == "u8":
        np.testing.assert_array_equal(out.astype(np.int64), ref, err_msg=what)
    else:
        assert_float_parity(out, ref, ab, what=what)


@pytest.mark.parametrize("dtype", ["f32", "u8", "bf16"])
def test_lofar_real_dms_every_fitting_variant(dtype):
    """LOFAR band, 96 trials (DM 0-23.75: several DM tiles of every shape),
    2 beams, 5000 output samples (a ragged last time tile): every CTA shape of
    the lane-strided and register-window kinds that fits, against the
    oracle. DM tiles of 8 or more trials must fit."""
    s = synth.setup("lofar").with_(n_dm=96, n_out=5000)
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    assert int(sh[1, 0] - sh[0, 0]) > 800  # one DM step moves channel 0 by > 800 samples
    s, x, w = _inputs(s, sh, dtype, 5, B=2)
    plan = Plan.from_setup(s)
    np.testing.assert_array_equal(plan.shifts(), sh)
    ref, ab = _reference(x, w, sh, s.n_out, dtype)
    xd, wd = to_dev(x, dtype), weights_dev(w, dtype)
    _check(plan.execute(xd, wd).cpu().numpy(), ref, ab, dtype, "default %s" % plan.variant)
    seen, ran, big_tiles = set(), 0, 0
    for v in variants():
        if v["kind"] not in (0, 1, 5) or v["stages"] == 4:
            continue
        key = (v["kind"], v["dm_per_thread"], v["samples_per_thread"], v["warps_dm"],
               v["warps_time"], v["chans_per_stage"])
        if key in seen:
            continue
        seen.add(key)
        try:
            plan.variant = v
        except DDError:
            continue  # the split windows of this shape do not fit shared memory
        _check(plan.execute(xd, wd).cpu().numpy(), ref, ab, dtype, str(v))
        ran += 1
        big_tiles += v["dm_per_thread"] * v["warps_dm"] >= 8
    assert ran >= 16 and big_tiles >= 5, (ran, big_tiles)
    plan.check_device()


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_coarse_dm_grid_low_band(dtype):
    """16 channels over 120-136 MHz at 64 us with DM steps of 60: adjacent
    trials' delays in the lowest channel differ by ~5.7e4 samples, which no
    union window can stage; the plan is accepted and matches the oracle,
    tuned variant included."""
    freqs = 120.0 + np.arange(16) * 1.0
    dms = np.arange(6) * 60.0
    sh = oracle.shift_table(freqs, freqs[-1], 64e-6, dms)
    assert int(sh[1, 0] - sh[0, 0]) > 50000
    S = 3000
    rng = np.random.default_rng(7)
    t_in = S + int(sh.max())
    stride = synth.padded_stride(t_in, dtype)
    xf = rng.standard_normal((1, 16, stride)).astype(np.float32)
    xf[:, :, t_in:] = np.nan
    w = rng.uniform(0.5, 1.5, 16).astype(np.float32)
    if dtype == "u8":
        x, w = synth.quantize_u8(np.nan_to_num(xf, nan=3.0)), synth.quantize_weights_q8(w)
    else:
        x = xf
    plan = Plan(freqs, freqs[-1], 64e-6, dms, S, batch=1, dtype=dtype)
    np.testing.assert_array_equal(plan.shifts(), sh)
    ref, ab = _reference(x, w, sh, S, dtype)
    xd, wd = to_dev(x, dtype), weights_dev(w, dtype)
    _check(plan.execute(xd, wd).cpu().numpy(), ref, ab, dtype, "default %s" % plan.variant)
    plan.tune(budget_ms=3000)
    _check(plan.execute(xd, wd).cpu().numpy(), ref, ab, dtype, "tuned %s" % plan.variant)
    plan.check_device()


def test_lofar_full_size_sampled():
    """The full LOFAR instance the benchmark times (32 channels, 2048 trials
    DM 0-511.75, 200000 samples = 1 s, FP32, weights U(0.5, 1.5) with 5 %
    masked) in its tuned variant: 4000 sampled outputs plus pulses and
    corners against the oracle."""
    s = synth.setup("lofar")
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    s, x, w = _inputs(s, sh, "f32", 8)
    plan = Plan.from_setup(s)
    plan.tune(budget_ms=6000)
    out = plan.execute(to_dev(x, "f32"), weights_dev(w, "f32"))
    torch.cuda.synchronize()
    pulses = synth.pulse_plan(s, 8, amp=(4.0, 8.0))
    rng = np.random.default_rng(24)
    n = 4000
    pd = np.concatenate([rng.integers(0, s.n_dm, n), [p[1] for p in pulses],
                         [0, s.n_dm - 1, s.n_dm - 1, 0]])
    pt = np.concatenate([rng.integers(0, s.n_out, n), [p[2] for p in pulses],
                         [0, s.n_out - 1, 0, s.n_out - 1]])
    pb = np.zeros_like(pd)
    got = out[0][torch.from_numpy(pd).cuda(), torch.from_numpy(pt).cuda()].cpu().numpy()
    ref, ab = points_by_beam(x, w, sh, pb, pd, pt, "f32")
    assert_float_parity(got, ref, ab, what="lofar %s" % plan.variant)
    plan.check_device()
    # a wide DM tile (its channel windows split per trial) on the same data
    plan.variant = dict(kind=0, dm_per_thread=4, samples_per_thread=4, warps_dm=2, warps_time=4,
                        chans_per_stage=4, stages=2)
    out = plan.execute(to_dev(x, "f32"), weights_dev(w, "f32"))
    got = out[0][torch.from_numpy(pd).cuda(), torch.from_numpy(pt).cuda()].cpu().numpy()
    assert_float_parity(got, ref, ab, what="lofar %s" % plan.variant)
    plan.check_device()


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_batch_with_a_wide_delay_plan(dtype):
    """One persistent launch over a LOFAR-band plan (per-trial staging
    windows, delays ~900 samples apart per DM step) and a 64-channel L-band
    plan (union windows), with their own tile shapes inside the launch:
    both match the oracle, before and after the batch tuner."""
    from paper_1601_05052_gb300 import Batch
    lo = synth.setup("lofar").with_(n_dm=64, n_out=3000)
    sh_lo = oracle.shift_table(lo.freqs(), lo.f_ref, lo.t_samp, lo.dms())
    hi = synth.setup("lband64").with_(n_out=3000)
    sh_hi = oracle.shift_table(hi.freqs(), hi.f_ref, hi.t_samp, hi.dms())
    lo, x_lo, w_lo = _inputs(lo, sh_lo, dtype, 8, B=2)
    hi, x_hi, w_hi = _inputs(hi, sh_hi, dtype, 9, B=3)
    plans = [Plan.from_setup(lo), Plan.from_setup(hi)]
    refs = [_reference(x_lo, w_lo, sh_lo, lo.n_out, dtype),
            _reference(x_hi, w_hi, sh_hi, hi.n_out, dtype)]
    xs = [to_dev(x_lo, dtype), to_dev(x_hi, dtype)]
    ws = [weights_dev(w_lo, dtype), weights_dev(w_hi, dtype)]
    batch = Batch(plans)
    for stage in ("configured", "tuned"):
        if stage == "tuned":
            batch.tune(budget_ms=3000)
        outs = batch.execute(xs, ws)
        for i, (out, (ref, ab)) in enumerate(zip(outs, refs)):
            _check(out.cpu().numpy(), ref, ab, dtype,
                   "%s plan %d %s" % (stage, i, batch.plan_variant(i)))
    for p in plans:
        p.check_device()
