"""GPU parity of the persistent, graph-replayed batched forward: uneven plans
in one launch, against the oracle (full on small batches, sampled and
bit-exact on the 96 + 32 beam 8-bit workload)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1601_05052_gb300 import Batch, Plan
from gpu_util import assert_float_parity, points_by_beam, random_case, to_dev, weights_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "u8", "bf16"])
def test_small_uneven_batch_full(dtype):
    rng = np.random.default_rng(31)
    shapes = [(3, 37, 29, 1000, 150), (2, 64, 70, 333, 900), (1, 5, 3, 2049, 20)]
    cases = [random_case(rng, *c, dtype=dtype) for c in shapes]
    plans = [Plan(shifts=sh, n_out=c[3], batch=c[0], dtype=dtype) for (sh, _, _), c in
             zip(cases, shapes)]
    batch = Batch(plans)
    xs = [to_dev(x, dtype) for (_, x, _) in cases]
    ws = [weights_dev(w, dtype) for (_, _, w) in cases]
    for rep in range(3):  # first call builds the graph args, later calls replay
        outs = batch.execute(xs, ws)
        for (sh, x, w), c, o in zip(cases, shapes, outs):
            o = o.cpu().numpy()
            if dtype == "u8":
                np.testing.assert_array_equal(o.astype(np.int64), oracle.forward_u8(x, w, sh, c[3]))
            else:
                ref, ab = oracle.forward(x, w, sh, c[3], dtype=dtype, with_absum=True)
                assert_float_parity(o, ref, ab, what="batch %s" % (c,))
    # new output buffers: the graph picks up the new pointers
    outs2 = [torch.zeros_like(o) for o in outs]
    batch.execute(xs, ws, outs2)
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)
    for p in plans:
        p.check_device()


def test_batched_96_plus_32_uneven_beams_u8_sampled():
    """96 beams of the 64-channel setup plus 32 low-frequency beams (256 ch
    over 120-180 MHz, 2000 trials, 10000 samples), 8-bit input, unit weights,
    one persistent launch: sampled outputs bit-exact, and the tuned batch
    variant stays exact."""
    hi, lo = synth.setup("lband64_x96_u8"), synth.setup("lowfreq256_u8")
    plans, data = [], []
    for s, seed in ((hi, 41), (lo, 42)):
        sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
        pulses = synth.pulse_plan(s, seed, amp=(3.0, 6.0))
        x = synth.make_input(s, sh, seed=seed, pulses=pulses)
        w = np.ones(s.n_chan, np.int32)
        plans.append(Plan.from_setup(s))
        data.append((s, sh, x, w))
    batch = Batch(plans)
    xs = [to_dev(d[2], "u8") for d in data]
    ws = [weights_dev(d[3], "u8") for d in data]
    rng = np.random.default_rng(4)
    for attempt in range(2):
        outs = batch.execute(xs, ws)
        torch.cuda.synchronize()
        for (s, sh, x, w), o in zip(data, outs):
            n = 3000
            pb = rng.integers(0, s.batch, n)
            pd = rng.integers(0, s.n_dm, n)
            pt = rng.integers(0, s.n_out, n)
            ref = oracle.forward_points_u8(x, w, sh, pb, pd, pt)
            got = o[torch.from_numpy(pb).cuda(), torch.from_numpy(pd).cuda(),
                    torch.from_numpy(pt).cuda()].cpu().numpy()
            np.testing.assert_array_equal(got.astype(np.int64), ref)
        if attempt == 0:
            rep = batch.tune(budget_ms=20000)
            assert rep["n_tried"] >= 1
    for p in plans:
        p.check_device()


def test_batched_96_plus_32_uneven_beams_f16_sampled():
    """The same 96 + 32 beam batch with 16-bit float input (FP32
    accumulation) in one persistent launch, as the benchmark times it: its
    default variant and the tuned one, 3000 sampled outputs per setup within
    1e-4 * sum|w*in| of the FP64 oracle."""
    hi, lo = synth.setup("lband64_x96_u8"), synth.setup("lowfreq256_u8")
    plans, data = [], []
    for s, seed in ((hi, 43), (lo, 44)):
        s = s.with_(dtype="f16")
        sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
        pulses = synth.pulse_plan(s, seed, amp=(3.0, 6.0))
        x = synth.make_input(s, sh, seed=seed, pulses=pulses)
        w = np.ones(s.n_chan, np.float32)
        plans.append(Plan.from_setup(s))
        data.append((s, sh, x, w))
    batch = Batch(plans)
    xs = [to_dev(d[2], "f16") for d in data]
    ws = [weights_dev(d[3], "f16") for d in data]
    rng = np.random.default_rng(6)
    for attempt in range(2):
        outs = batch.execute(xs, ws)
        torch.cuda.synchronize()
        for (s, sh, x, w), o in zip(data, outs):
            n = 3000
            pb = rng.integers(0, s.batch, n)
            pd = rng.integers(0, s.n_dm, n)
            pt = rng.integers(0, s.n_out, n)
            ref, ab = points_by_beam(x, w, sh, pb, pd, pt, "f16")
            got = o[torch.from_numpy(pb).cuda(), torch.from_numpy(pd).cuda(),
                    torch.from_numpy(pt).cuda()].cpu().numpy()
            assert_float_parity(got, ref, ab, what="f16 batch %s, attempt %d" % (s.name, attempt))
        if attempt == 0:
            batch.tune(budget_ms=15000)
    for p in plans:
        p.check_device()


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_per_plan_tile_shapes_in_one_launch(dtype):
    """Each plan of a batch keeps its own split of the trial warps (its DM x
    time tile) and its own chunk size inside the one persistent launch; the
    results stay exact, and a variant that does not share the launch's
    kernel, staging depth or warp count is refused without changing any."""
    from paper_1601_05052_gb300 import DDError, compute_shifts
    rng = np.random.default_rng(33)
    cases, plans = [], []
    # three uneven Eq. 1 tables (the sub-band kinds fit them)
    for C, D, S, f0, bw in ((48, 64, 700, 1250.0, 300.0), (32, 40, 1500, 1400.0, 100.0),
                            (20, 24, 900, 1300.0, 200.0)):
        freqs = f0 + np.arange(C) * (bw / C)
        sh = compute_shifts(freqs, freqs[-1], 100e-6, np.arange(D) * 0.25).astype(np.int64)
        t_in = S + int(sh.max())
        x = rng.standard_normal((2, C, synth.padded_stride(t_in, dtype))).astype(np.float32)
        w = rng.uniform(0.5, 1.5, C).astype(np.float32)
        if dtype == "u8":
            x, w = synth.quantize_u8(x), synth.quantize_weights_q8(w)
        cases.append((sh, x, w, S))
    plans = [Plan(shifts=c[0], n_out=c[3], batch=c[1].shape[0], dtype=dtype) for c in cases]
    batch = Batch(plans)
    xs = [to_dev(c[1], dtype) for c in cases]
    ws = [weights_dev(c[2], dtype) for c in cases]

    def check(what):
        outs = batch.execute(xs, ws)
        for (sh, x, w, S), o in zip(cases, outs):
            o = o.cpu().numpy()
            if dtype == "u8":
                np.testing.assert_array_equal(o.astype(np.int64), oracle.forward_u8(x, w, sh, S),
                                              err_msg=what)
            else:
                ref, ab = oracle.forward(x, w, sh, S, dtype=dtype, with_absum=True)
                assert_float_parity(o, ref, ab, what=what)

    tried = 0
    for kind, dpt, spt, tw in ((0, 4, 4, 8), (2, 4, 8, 8), (4, 4, 8, 16), (5, 4, 8, 8)):
        base = dict(kind=kind, dm_per_thread=dpt, samples_per_thread=spt, warps_dm=2,
                    warps_time=tw // 2, chans_per_stage=4, stages=2)
        try:
            batch.variant = base
        except DDError:
            continue  # a plan has too many delay patterns per DM tile for this sub-band shape
        combos = [(wd, tw // wd, c) for wd in (1, 2, 4, 8, 16) if wd <= tw and tw % wd == 0
                  for c in (4, 8, 16)]
        for i in range(len(plans)):
            # the first other shape (from a start that differs per plan) that fits plan i
            for k in range(len(combos)):
                wd, wt, c = combos[(5 * i + k) % len(combos)]
                v = dict(base, warps_dm=wd, warps_time=wt, chans_per_stage=c)
                if v == base:
                    continue
                try:
                    batch.set_plan_variant(i, v)
                except DDError:
                    continue  # does not fit (e.g. a sub-band DM tile not a multiple of 8)
                assert batch.plan_variant(i) == v
                break
        pv = batch.plan_variants
        assert len({tuple(sorted(v.items())) for v in pv}) >= 2, pv  # shapes differ per plan
        check("per-plan shapes, kind %d: %s" % (kind, pv))
        tried += 1
        before = batch.plan_variants
        with pytest.raises(DDError):
            batch.set_plan_variant(0, dict(base, stages=3))
        with pytest.raises(DDError):
            batch.set_plan_variant(1, dict(base, warps_dm=1, warps_time=1))
        assert batch.plan_variants == before
        check("after refused changes, kind %d" % kind)
    assert tried == 4
    for p in plans:
        p.check_device()


@pytest.mark.parametrize("kind", [0, 5])
def test_batch_tiles_with_fewer_chunks_than_stages(kind):
    """Plans of 16 channels staged 16 at a time have one chunk per tile, fewer
    than the staging depth, so a CTA's staging warp never waits for the
    others and can reach the next work item first; every tile of many must
    still be summed exactly once (8-bit input, exact)."""
    rng = np.random.default_rng(60 + kind)
    cases, plans = [], []
    for B, D, S in ((40, 64, 3000), (24, 32, 1000)):
        sh = np.sort(rng.integers(0, 200, size=(D, 16)), axis=0)
        x = rng.integers(0, 256, size=(B, 16, synth.padded_stride(S + int(sh.max()), "u8")),
                         dtype=np.uint8)
        w = rng.integers(-300, 300, size=16).astype(np.int32)
        cases.append((sh, x, w, S))
        plans.append(Plan(shifts=sh, n_out=S, batch=B, dtype="u8"))
    batch = Batch(plans)
    batch.variant = dict(kind=kind, dm_per_thread=4, samples_per_thread=8, warps_dm=4,
                         warps_time=2, chans_per_stage=16, stages=3)
    xs = [to_dev(c[1], "u8") for c in cases]
    ws = [weights_dev(c[2], "u8") for c in cases]
    for _ in range(3):
        outs = batch.execute(xs, ws)
        for (sh, x, w, S), o in zip(cases, outs):
            np.testing.assert_array_equal(o.cpu().numpy().astype(np.int64),
                                          oracle.forward_u8(x, w, sh, S))
    for p in plans:
        p.check_device()

