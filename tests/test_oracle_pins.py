"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own code (hand-worked fixtures, closed forms,
special cases, algebraic identities, brute force on tiny inputs)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
K_PAPER = 4150.0      # Eq. 1 as printed in the paper (approximate constant)
K_PRECISE = 4.148808e3


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- shift table (Eq. 1)

def test_shift_hand_worked_cases():
    g = _gold("shift_hand.json")
    for case in g["cases"]:
        got = oracle.shift_table(case["freqs"], case["f_ref"], case["t_samp"], case["dm"])
        assert got.tolist() == case["expected"], case["_derivation"]


@pytest.mark.parametrize("name", ["lband64", "apertif_survey", "diff16_512ch", "lowfreq256_u8", "lofar"])
def test_shift_table_structure(name):
    s = synth.setup(name)
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    assert sh.shape == (s.n_dm, s.n_chan)
    assert (sh[0] == 0).all(), "DM 0 row must be all zeros"
    assert (sh[:, -1] == 0).all(), "the reference (top) channel has no delay"
    assert (np.diff(sh, axis=0) >= 0).all(), "delay non-decreasing in DM"
    assert (np.diff(sh, axis=1) <= 0).all(), "delay non-increasing in frequency"


def test_shift_scale_matches_paper_constant():
    """Eq. 1 with the paper's printed K ~ 4150 agrees to K's precision
    (0.029 %) plus one rounding step: pins units (MHz, seconds) and the
    inverse-square law's scale."""
    s = synth.setup("apertif_survey")
    f, fr, ts, dm = s.freqs(), s.f_ref, s.t_samp, s.dms()
    sh = oracle.shift_table(f, fr, ts, dm)
    approx = K_PAPER * dm[:, None] * (1 / f[None, :] ** 2 - 1 / fr ** 2) / ts
    rel = abs(K_PAPER - K_PRECISE) / K_PRECISE
    assert (np.abs(sh - approx) <= rel * approx + 1.0).all()


def test_shift_linear_in_dm_and_inverse_in_tsamp():
    s = synth.setup("diff16_512ch")
    f, fr = s.freqs(), s.f_ref
    dm = np.array([10.0, 20.0, 40.0])
    a = oracle.shift_table(f, fr, 1e-4, dm)
    # doubling DM doubles the unrounded delay: rounded values differ by <= 1
    assert (np.abs(a[1] - 2 * a[0]) <= 1).all() and (np.abs(a[2] - 2 * a[1]) <= 1).all()
    b = oracle.shift_table(f, fr, 0.5e-4, dm)
    assert (np.abs(b - 2 * a) <= 1).all()


def test_shift_inverse_square_law():
    """With f_ref -> infinity the delay is proportional to f^-2."""
    f = np.array([100.0, 200.0, 400.0])
    sh = oracle.shift_table(f, 1e12, 1e-6, [1000.0])[0]
    assert abs(sh[0] / sh[1] - 4.0) < 1e-6 and abs(sh[1] / sh[2] - 4.0) < 1e-5


def test_shift_rejects_negative_and_bad_args():
    with pytest.raises(ValueError):
        oracle.shift_table([1500.0, 1400.0], 1400.0, 1e-4, [10.0])  # channel above f_ref
    with pytest.raises(ValueError):
        oracle.shift_table([1400.0], 1400.0, 0.0, [1.0])


def test_paper_flop_count_per_dm():
    """Section IV: the Apertif setup is 20 MFLOP per DM, LOFAR 6 MFLOP per DM
    (one addition per channel per output sample)."""
    ap, lo = synth.setup("apertif_survey"), synth.setup("lofar")
    assert ap.n_out * ap.n_chan == 20_480_000
    assert lo.n_out * lo.n_chan == 6_400_000


# ---------------------------------------------------------------- forward (Algorithm 1)

def _tiny():
    g = _gold("tiny_forward.json")
    x = np.array(g["input"], dtype=np.float32)[None]
    return g, x, np.array(g["weights"], np.float32), np.array(g["shifts"], np.int64)


def test_forward_tiny_hand_worked():
    g, x, w, sh = _tiny()
    out = oracle.forward(x, w, sh, g["n_out"])
    assert out[0].tolist() == g["expected_out"]


def test_forward_u8_tiny_hand_worked():
    g, x, w, sh = _tiny()
    xs = (x[:, :, :] // 10).astype(np.uint8)  # rows 0,1,2,3..; 1..6; 10..60
    out = oracle.forward_u8(xs, np.array([1, 2, 3]), sh, g["n_out"])
    ref = [[sum(int(w_) * int(xs[0, c, t + sh[d, c]]) for c, w_ in enumerate([1, 2, 3]))
            for t in range(4)] for d in range(2)]
    assert out[0].tolist() == ref


def _rand_case(rng, B=2, C=5, D=4, S=9, max_shift=6, dtype="f32"):
    sh = np.sort(rng.integers(0, max_shift + 1, size=(D, C)), axis=0)
    stride = synth.padded_stride(S + max_shift, dtype)
    x = rng.standard_normal((B, C, stride)).astype(np.float32)
    w = rng.uniform(-1, 2, size=C).astype(np.float32)
    return sh, x, w, stride


def test_forward_brute_force_python_loops():
    rng = np.random.default_rng(11)
    for _ in range(5):
        sh, x, w, stride = _rand_case(rng)
        B, C, _ = x.shape
        D, S = sh.shape[0], 9
        out = oracle.forward(x, w, sh, S)
        for b, d, t in itertools.product(range(B), range(D), range(S)):
            ref = 0.0
            for c in range(C):
                ref += float(w[c]) * float(x[b, c, t + sh[d, c]])
            assert out[b, d, t] == pytest.approx(ref, rel=1e-14, abs=1e-14)


def test_forward_dm0_is_weighted_channel_sum():
    """Section IV-C: with every trial DM equal to 0 there are no shifts and
    every output row is the (weighted) channel sum."""
    s = synth.setup("lband64")
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, np.zeros(8))
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, s.n_chan, 512)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, s.n_chan)
    out = oracle.forward(x, w, sh, 512)
    ref = np.einsum("c,ct->t", w, x[0].astype(np.float64))
    for d in range(8):
        np.testing.assert_allclose(out[0, d], ref, rtol=1e-12, atol=1e-12)


def test_forward_constant_and_ramp_closed_forms():
    s = synth.setup("lband64")
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    S = 300
    T = S + int(sh.max())
    w = np.linspace(0.25, 2.0, s.n_chan)
    const = np.full((1, s.n_chan, T), 3.0, np.float32)
    out = oracle.forward(const, w, sh, S)
    np.testing.assert_allclose(out, 3.0 * w.sum(), rtol=1e-13)
    ramp = np.broadcast_to(np.arange(T, dtype=np.float32), (1, s.n_chan, T)).copy()
    out = oracle.forward(ramp, w, sh, S)
    t = np.arange(S)
    ref = t[None, :] * w.sum() + (sh * w[None, :]).sum(1)[:, None]
    np.testing.assert_allclose(out[0], ref, rtol=1e-13)


def test_forward_dispersed_impulse_peaks_at_its_trial():
    """A unit impulse dispersed along trial d* sums to sum_c w_c exactly at
    (d*, t0); any other trial reaching that value must share d*'s shift column
    on every weighted channel."""
    s = synth.setup("lband64")
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    S, dstar, t0 = 2048, 40, 1000
    T = S + int(sh.max())
    w = synth.make_weights(s.n_chan, 5, "uniform")
    x = np.zeros((1, s.n_chan, T), np.float32)
    x[0, np.arange(s.n_chan), t0 + sh[dstar]] = 1.0
    out = oracle.forward(x, w, sh, S)[0]
    peak = w.astype(np.float64).sum()
    assert out[dstar, t0] == pytest.approx(peak, rel=1e-14)
    assert out.max() == pytest.approx(peak, rel=1e-14)
    wmask = w != 0
    for d, t in zip(*np.nonzero(np.isclose(out, peak, rtol=1e-12))):
        assert t == t0 and (sh[d, wmask] == sh[dstar, wmask]).all()


def test_forward_linearity_and_time_shift():
    rng = np.random.default_rng(5)
    sh, x, w, stride = _rand_case(rng, B=1, C=7, D=5, S=12, max_shift=9)
    y = rng.standard_normal(x.shape).astype(np.float32)
    a, b = 0.75, -2.5
    lhs = oracle.forward(a * x.astype(np.float64) + b * y.astype(np.float64), w, sh, 12)
    rhs = a * oracle.forward(x, w, sh, 12) + b * oracle.forward(y, w, sh, 12)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    # advancing the input by one sample advances every output series by one
    x1 = np.roll(x, -1, axis=2)
    o0 = oracle.forward(x, w, sh, 12)
    o1 = oracle.forward(x1, w, sh, 11)
    np.testing.assert_array_equal(o1[:, :, :11], o0[:, :, 1:12])


def test_forward_u8_matches_exact_integer_sum_and_constant():
    rng = np.random.default_rng(9)
    sh = np.sort(rng.integers(0, 40, size=(6, 8)), axis=0)
    S = 50
    x = rng.integers(0, 256, size=(2, 8, synth.padded_stride(S + 40, "u8"))).astype(np.uint8)
    wq = rng.integers(0, 385, size=8)
    out = oracle.forward_u8(x, wq, sh, S)
    # the float64 path sums the same small integers exactly
    ref = oracle.forward(x.astype(np.float32), wq.astype(np.float64), sh, S)
    assert (out == ref.astype(np.int64)).all()
    const = np.full_like(x, 255)
    assert (oracle.forward_u8(const, wq, sh, S) == 255 * wq.sum()).all()


def test_forward_points_u8_agree_with_full():
    rng = np.random.default_rng(12)
    sh = np.sort(rng.integers(0, 30, size=(5, 7)), axis=0)
    x = rng.integers(0, 256, size=(3, 7, synth.padded_stride(20 + 30, "u8"))).astype(np.uint8)
    wq = rng.integers(-5, 400, size=7)
    full = oracle.forward_u8(x, wq, sh, 20)
    pb, pd, pt = rng.integers(0, 3, 50), rng.integers(0, 5, 50), rng.integers(0, 20, 50)
    np.testing.assert_array_equal(oracle.forward_points_u8(x, wq, sh, pb, pd, pt), full[pb, pd, pt])


def test_forward_points_agree_with_full():
    rng = np.random.default_rng(2)
    sh, x, w, stride = _rand_case(rng, B=3, C=6, D=5, S=10, max_shift=7)
    full, ab = oracle.forward(x, w, sh, 10, with_absum=True)
    pb, pd, pt = rng.integers(0, 3, 40), rng.integers(0, 5, 40), rng.integers(0, 10, 40)
    v, a = oracle.forward_points(x, w, sh, pb, pd, pt)
    np.testing.assert_array_equal(v, full[pb, pd, pt])
    np.testing.assert_array_equal(a, ab[pb, pd, pt])
    assert (ab >= np.abs(full) - 1e-12).all()


def test_decode_bf16_and_f16():
    bits = np.array([0x3F80, 0xC000, 0x0000, 0x3E80], np.uint16)  # 1, -2, 0, 0.25
    assert oracle.decode(bits, "bf16").tolist() == [1.0, -2.0, 0.0, 0.25]
    h = np.array([1.5, -0.125], np.float16)
    assert oracle.decode(h, "f16").tolist() == [1.5, -0.125]


# ---------------------------------------------------------------- adjoint and grad_w

def test_adjoint_tiny_hand_worked():
    g, x, w, sh = _tiny()
    cot = np.zeros((1, 2, 4))
    d, t = g["adjoint_unit_at"]
    cot[0, d, t] = 1.0
    gin = oracle.adjoint(cot, w, sh, g["t_in"])
    exp = np.zeros((1, 3, g["t_in"]))
    for c, tau, v in g["expected_gin_nonzero"]:
        exp[0, c, tau] = v
    np.testing.assert_array_equal(gin, exp)
    gw = oracle.grad_w(np.ones((1, 2, 4)), x, sh)
    assert gw.tolist() == g["expected_grad_w_ones"]


def test_adjoint_identity():
    """<A x, y> = <x, A^T y> for random x, y (the defining property)."""
    rng = np.random.default_rng(21)
    for _ in range(3):
        sh, x, w, stride = _rand_case(rng, B=2, C=9, D=7, S=33, max_shift=20)
        y = rng.standard_normal((2, 7, 33))
        lhs = float((oracle.forward(x, w, sh, 33) * y).sum())
        rhs = float((x.astype(np.float64) * oracle.adjoint(y, w, sh, stride)).sum())
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_adjoint_points_agree_with_scatter():
    rng = np.random.default_rng(4)
    sh, x, w, stride = _rand_case(rng, B=2, C=6, D=5, S=11, max_shift=8)
    y = rng.standard_normal((2, 5, 11))
    full = oracle.adjoint(y, w, sh, stride)
    pb, pc, pt = rng.integers(0, 2, 60), rng.integers(0, 6, 60), rng.integers(0, 11 + 8, 60)
    v, _ = oracle.adjoint_points(y, w, sh, pb, pc, pt)
    np.testing.assert_allclose(v, full[pb, pc, pt], rtol=1e-13, atol=1e-13)


def test_grad_w_central_difference():
    """<g, out(w)> is linear in w, so a central difference is exact up to
    rounding for any step."""
    rng = np.random.default_rng(8)
    sh, x, w, stride = _rand_case(rng, B=2, C=5, D=4, S=16, max_shift=10)
    y = rng.standard_normal((2, 4, 16))
    gw = oracle.grad_w(y, x, sh)
    h = 1e-3
    for c in range(5):
        wp, wm = w.astype(np.float64).copy(), w.astype(np.float64).copy()
        wp[c] += h
        wm[c] -= h
        fd = ((oracle.forward(x, wp, sh, 16) * y).sum() - (oracle.forward(x, wm, sh, 16) * y).sum()) / (2 * h)
        assert gw[c] == pytest.approx(fd, rel=1e-8, abs=1e-9)
    sel = np.array([4, 0, 2])
    v, _ = oracle.grad_w_channels(y, x, sh, sel)
    np.testing.assert_allclose(v, gw[sel], rtol=1e-13)


def test_input_recipe_places_pulses_on_the_trial():
    """The synthetic recipe: a pulse added along trial d* dominates trial d*
    at t0 (noise N(0,1), amplitude 5, 64 channels)."""
    s = synth.setup("lband64")
    sh = oracle.shift_table(s.freqs(), s.f_ref, s.t_samp, s.dms())
    pulses = synth.pulse_plan(s, 1, fixed=(40, 1000, 5.0))
    x = synth.make_input(s, sh, seed=1, pulses=pulses)
    assert np.isnan(x[0, 0, s.n_out + int(sh.max()):]).all()
    out = oracle.forward(x, np.ones(s.n_chan), sh, s.n_out)[0]
    d, t = np.unravel_index(np.argmax(out), out.shape)
    assert t == 1000 and abs(int(d) - 40) <= 1
