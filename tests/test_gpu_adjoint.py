"""GPU parity of the adjoint (grad_in, gather form) and grad_w kernels against
the oracle's scatter transpose, the adjoint identity, autograd wiring, and
the differentiable workload (16 beams, 512 ch, 1024 trials, 8192 samples)
against FP64 central finite differences."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1601_05052_gb300 import Plan, dedisperse
from gpu_util import assert_float_parity, random_case, to_dev, weights_dev

pytestmark = pytest.mark.gpu

CASES = [  # (B, C, D, S, max_shift)
    (2, 37, 29, 1000, 150),
    (1, 5, 70, 333, 900),
    (3, 20, 3, 257, 20),
    (1, 1, 1, 1, 0),
]


@pytest.mark.parametrize("case", CASES)
def test_adjoint_and_grad_w_match_oracle(case):
    B, C, D, S, ms = case
    rng = np.random.default_rng(1000 + C)
    sh, x, w = random_case(rng, B, C, D, S, ms, "f32")
    x = np.nan_to_num(x, nan=0.0)  # grad_w reads only [0, T_in); keep pad finite for the oracle
    g = rng.standard_normal((B, D, S)).astype(np.float32)
    plan = Plan(shifts=sh, n_out=S, batch=B)
    gin, gw = plan.adjoint(to_dev(g, "f32"), weights_dev(w, "f32"), to_dev(x, "f32"))
    stride = plan.input_stride
    ref = oracle.adjoint(g, w, sh, stride)
    ab = oracle.adjoint(np.abs(g), np.abs(w), sh, stride)
    assert_float_parity(gin.cpu().numpy(), ref, ab, what="grad_in")
    refw = oracle.grad_w(g, x, sh)
    abw = oracle.grad_w(np.abs(g), np.abs(x), sh)
    assert_float_parity(gw.cpu().numpy(), refw, abw, what="grad_w")
    # deterministic: a second call gives identical bits
    gin2, gw2 = plan.adjoint(to_dev(g, "f32"), weights_dev(w, "f32"), to_dev(x, "f32"))
    assert torch.equal(gin, gin2) and torch.equal(gw, gw2)
    plan.check_device()


def test_adjoint_every_kernel_kind_with_zero_borders():
    """The adjoint's transposed gather skips the chunks whose staged windows
    lie wholly in the cotangent's zero borders. Every kernel kind and CTA
    shape that fits the transposed plan must still match the oracle: an Eq. 1
    table (48 channels over 1250-1550 MHz, 100 us, 96 trials of step 0.25)
    with fewer output samples than its largest delay, so that whole time
    tiles at both ends have no live chunk at all."""
    from paper_1601_05052_gb300 import DDError, compute_shifts, variants
    C, D, B = 48, 96, 2
    freqs = 1250.0 + np.arange(C) * (300.0 / C)
    sh = compute_shifts(freqs, freqs[-1], 100e-6, np.arange(D) * 0.25).astype(np.int64)
    S = int(sh.max()) - 37
    rng = np.random.default_rng(21)
    plan = Plan(shifts=sh, n_out=S, batch=B)
    x = rng.standard_normal(plan.in_shape).astype(np.float32)
    w = rng.uniform(-0.5, 1.5, C).astype(np.float32)
    g = rng.standard_normal((B, D, S)).astype(np.float32)
    stride = plan.input_stride
    ref = oracle.adjoint(g, w, sh, stride)
    ab = oracle.adjoint(np.abs(g), np.abs(w), sh, stride)
    refw = oracle.grad_w(g, x, sh)
    abw = oracle.grad_w(np.abs(g), np.abs(x), sh)
    gd, wd, xd = to_dev(g, "f32"), weights_dev(w, "f32"), to_dev(x, "f32")
    seen, kinds = set(), {}
    for v in variants():
        key = (v["kind"], v["dm_per_thread"], v["samples_per_thread"], v["warps_dm"],
               v["warps_time"], v["chans_per_stage"])
        if key in seen or v["stages"] == 4:
            continue
        seen.add(key)
        try:
            plan.adjoint_variant = v
        except DDError:
            continue  # does not fit the transposed plan
        assert plan.adjoint_variant == v
        gin, gw = plan.adjoint(gd, wd, xd)
        assert_float_parity(gin.cpu().numpy(), ref, ab, what="grad_in %s" % v)
        assert_float_parity(gw.cpu().numpy(), refw, abw, what="grad_w %s" % v)
        kinds[v["kind"]] = kinds.get(v["kind"], 0) + 1
    assert all(kinds.get(k, 0) >= 2 for k in range(6)), kinds
    plan.check_device()


def test_adjoint_identity_on_gpu():
    rng = np.random.default_rng(3)
    sh, x, w = random_case(rng, 2, 48, 40, 2000, 500, "f32")
    x = np.nan_to_num(x, nan=0.0)
    y = rng.standard_normal((2, 40, 2000)).astype(np.float32)
    plan = Plan(shifts=sh, n_out=2000, batch=2)
    ax = plan.execute(to_dev(x, "f32"), weights_dev(w, "f32")).double()
    aty, _ = plan.adjoint(to_dev(y, "f32"), weights_dev(w, "f32"), need_gw=False)
    lhs = float((ax * torch.from_numpy(y).cuda().double()).sum())
    rhs = float((torch.from_numpy(x).cuda().double() * aty.double()).sum())
    assert lhs == pytest.approx(rhs, rel=1e-5)


def test_autograd_function_backward():
    rng = np.random.default_rng(4)
    sh, x, w = random_case(rng, 1, 16, 12, 300, 60, "f32")
    x = np.nan_to_num(x, nan=0.0)
    plan = Plan(shifts=sh, n_out=300, batch=1)
    xt = to_dev(x, "f32").requires_grad_(True)
    wt = weights_dev(w, "f32").requires_grad_(True)
    out = dedisperse(plan, xt, wt)
    g = torch.randn_like(out)
    out.backward(g)
    ref_gin = oracle.adjoint(g.cpu().numpy(), w, sh, plan.input_stride)
    ab = oracle.adjoint(np.abs(g.cpu().numpy()), np.abs(w), sh, plan.input_stride)
    assert_float_parity(xt.grad.cpu().numpy(), ref_gin, ab, what="autograd grad_in")
    ref_gw = oracle.grad_w(g.cpu().numpy(), x, sh)
    abw = oracle.grad_w(np.abs(g.cpu().numpy()), np.abs(x), sh)
    assert_float_parity(wt.grad.cpu().numpy(), ref_gw, abw, what="autograd grad_w")


def test_16beam_512ch_1024dm_finite_differences():
    """Loss = sum of out^2 over trials [256, 768) x samples [2048, 6144) of all
    16 beams; 32 input and 32 weight coordinates against FP64 central
    differences (h = 1e-3) of the oracle's loss restricted to the outputs each
    perturbation touches (exact for a quadratic loss)."""
    s = synth.setup("diff16_512ch")
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    pulses = synth.pulse_plan(s, 5)
    x = synth.make_input(s, sh, seed=5, pulses=pulses, pad_value=np.float32(0))
    w = synth.make_weights(s.n_chan, 5, "ones")
    D0, D1, T0, T1 = 256, 768, 2048, 6144
    plan = Plan.from_setup(s)
    xt = to_dev(x, "f32").requires_grad_(True)
    wt = weights_dev(w, "f32").requires_grad_(True)
    out = dedisperse(plan, xt, wt)
    loss = (out[:, D0:D1, T0:T1] ** 2).sum()
    loss.backward()
    gx, gw = xt.grad, wt.grad
    rng = np.random.default_rng(55)
    h = 1e-3

    def loss_terms(o):  # o: float64 outputs in the window
        return (o ** 2).sum()

    # input coordinates: perturbing in[b][c][tau] moves out[b][d][tau - shift[d][c]] by w_c*h
    n_in = 0
    while n_in < 32:
        b, c = int(rng.integers(0, s.batch)), int(rng.integers(0, s.n_chan))
        tau = int(rng.integers(T0, T1))
        ds = np.arange(D0, D1)
        ts = tau - sh[D0:D1, c]
        keep = (ts >= T0) & (ts < T1)
        if not keep.any():
            continue
        ds, ts = ds[keep], ts[keep]
        o, _ = oracle.forward_points(x, w, sh, np.full(ds.size, b), ds, ts)
        fd = (loss_terms(o + w[c] * h) - loss_terms(o - w[c] * h)) / (2 * h)
        got = float(gx[b, c, tau])
        assert got == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(2 * o * w[c]).sum() + 1e-6)
        n_in += 1
    # weight coordinates: perturbing w_c moves every window output by h * in[b][c][t + shift]
    chans = rng.choice(s.n_chan, 32, replace=False)
    bb, dd, tt = np.meshgrid(np.arange(s.batch), np.arange(D0, D1), np.arange(T0, T1),
                             indexing="ij")
    bb, dd, tt = bb.ravel(), dd.ravel(), tt.ravel()
    o, _ = oracle.forward_points(x, w, sh, bb, dd, tt)
    for c in chans:
        xc = x[bb, c, tt + sh[dd, c]].astype(np.float64)
        fd = (loss_terms(o + h * xc) - loss_terms(o - h * xc)) / (2 * h)
        got = float(gw[c])
        assert got == pytest.approx(fd, rel=1e-3, abs=1e-4 * np.abs(2 * o * xc).sum())
    plan.check_device()
