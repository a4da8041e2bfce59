"""Helpers shared by the GPU parity tests: uploads, oracle comparisons and the
per-output float tolerance |gpu - oracle| <= 1e-4 * sum_c |w_c * in| (the
FP32 summation bound over up to ~1600 terms, gamma_n ~ n * 2^-24, stays below
it), bit-exact equality for 8-bit input."""
import numpy as np
import torch

import oracle
import synth

REL_TOL = 1e-4


def to_dev(x: np.ndarray, dtype: str) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype == "bf16":
        t = t.view(torch.bfloat16)
    return t.cuda()


def weights_dev(w: np.ndarray, dtype: str) -> torch.Tensor:
    if dtype == "u8":
        return torch.from_numpy(np.ascontiguousarray(w, dtype=np.int32)).cuda()
    return torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda()


def assert_float_parity(got, ref, absum, rel=REL_TOL, what=""):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    bound = rel * absum
    bad = err > bound
    if bad.any():
        i = np.argmax(err - bound)
        raise AssertionError("%s: %d of %d outputs beyond tolerance; worst err %.3g vs bound %.3g "
                             "(flat index %d)" % (what, int(bad.sum()), bad.size, err.flat[i],
                                                  bound.flat[i], i))


def check_full(plan, x, w, shifts, dtype, what=""):
    """Runs the plan on (x, w) and compares every output with the oracle."""
    out = plan.execute(to_dev(x, dtype), weights_dev(w, dtype)).cpu().numpy()
    if dtype == "u8":
        ref = oracle.forward_u8(x, w, shifts, plan.n_out)
        np.testing.assert_array_equal(out.astype(np.int64), ref, err_msg=what)
    else:
        ref, ab = oracle.forward(x, w, shifts, plan.n_out, dtype=dtype, with_absum=True)
        assert_float_parity(out, ref, ab, what=what)
    return out


def random_case(rng, B, C, D, S, max_shift, dtype, monotone=True, weights="uniform"):
    if max_shift == 0:
        sh = np.zeros((D, C), np.int64)
    elif monotone:
        sh = np.sort(rng.integers(0, max_shift + 1, size=(D, C)), axis=0)
        sh[-1, 0] = max_shift
    else:
        sh = rng.integers(0, max_shift + 1, size=(D, C))
    t_in = S + int(sh.max())
    stride = synth.padded_stride(t_in, dtype)
    xf = rng.standard_normal((B, C, stride)).astype(np.float32)
    xf[:, :, t_in:] = np.nan  # pad entries must never reach an output
    if dtype == "f32":
        x = xf
    elif dtype == "f16":
        x = xf.astype(np.float16)
    elif dtype == "bf16":
        x = synth.to_bf16_bits(xf)
    else:
        x = synth.quantize_u8(np.nan_to_num(xf, nan=7.0))
    if weights == "ones":
        w = np.ones(C, np.float32)
    else:
        w = rng.uniform(-0.5, 1.5, C).astype(np.float32)
        w[rng.random(C) < 0.1] = 0.0
    if dtype == "u8":
        w = synth.quantize_weights_q8(w)
    return sh, x, w


def points_by_beam(x, w, sh, pb, pd, pt, dtype):
    """The oracle at sampled points, one beam at a time (a float beam decodes
    to FP64 on its own, so large batches never decode whole)."""
    if dtype == "u8":
        return oracle.forward_points_u8(x, w, sh, pb, pd, pt), None
    ref = np.empty(pb.size)
    ab = np.empty(pb.size)
    for b in np.unique(pb):
        m = pb == b
        ref[m], ab[m] = oracle.forward_points(x[b:b + 1], w, sh, np.zeros(m.sum(), np.int64),
                                              pd[m], pt[m], dtype=dtype)
    return ref, ab
