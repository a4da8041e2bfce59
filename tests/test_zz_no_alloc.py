"""dd_grad_w_noalloc: the weight gradient for callers that cannot allocate
device memory when they need it (their allocator already holds all free
memory, or allocation would stall a real-time stream). It must give the same
gradient as dd_adjoint and as the FP64 oracle, call after call, although
every call reuses one fixed device array for its partial sums. This file is
collected last so that a failure here stops a run only after every other
test has run."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1601_05052_gb300 import Plan, _lib
from gpu_util import assert_float_parity, random_case, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(plan, g, x):
    gw = torch.full((plan.n_chan,), float("nan"), dtype=torch.float32, device="cuda")
    lib = _lib.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(lib.dd_grad_w_noalloc(plan._h, ctypes.c_void_p(g.data_ptr()),
                                     ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(gw.data_ptr()),
                                     st))
    return gw


@pytest.mark.parametrize("case", [(2, 37, 29, 1000, 150), (3, 130, 70, 2049, 900)])
def test_noalloc_grad_w_matches_adjoint_twice(case):
    B, C, D, S, ms = case
    rng = np.random.default_rng(500 + C)
    sh, x0, w = random_case(rng, B, C, D, S, ms, "f32")
    plan = Plan(shifts=sh, n_out=S, batch=B)
    for call in range(2):  # two calls in a row, new data each time
        x = np.nan_to_num(x0, nan=0.0) if call == 0 else \
            rng.standard_normal(plan.in_shape).astype(np.float32)
        g = rng.standard_normal((B, D, S)).astype(np.float32)
        gd, xd = to_dev(g, "f32"), to_dev(x, "f32")
        got = _noalloc(plan, gd, xd)
        _, ref = plan.adjoint(gd, None, xd, need_gin=False, need_gw=True)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        # against the FP64 oracle, with the bound of the float tolerance
        exact = oracle.grad_w(g, x, sh)
        absum = oracle.grad_w(np.abs(g), np.abs(x), sh)
        assert_float_parity(got.cpu().numpy(), exact, absum, what="oracle, call %d" % call)
        # against dd_adjoint's weight gradient (both within the tolerance of
        # the exact value, so within twice it of each other)
        assert_float_parity(got.cpu().numpy(), ref.cpu().numpy().astype(np.float64), absum,
                            rel=2e-4, what="dd_adjoint, call %d" % call)
        again = _noalloc(plan, gd, xd)
        assert torch.equal(got, again)  # deterministic, stale scratch has no effect


def test_noalloc_rejects_oversized_and_non_f32_plans():
    lib = _lib.load()
    big = Plan(shifts=np.zeros((1, 4097), np.int32), n_out=8, batch=1)
    g = torch.zeros(big.out_shape, device="cuda")
    x = torch.zeros(big.in_shape, device="cuda")
    gw = torch.zeros(big.n_chan, device="cuda")
    st = lib.dd_grad_w_noalloc(big._h, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(gw.data_ptr()), None)
    assert st == 1 and b"4096" in lib.dd_last_error_message()
    u8 = Plan(shifts=np.zeros((1, 4), np.int32), n_out=8, batch=1, dtype="u8")
    st = lib.dd_grad_w_noalloc(u8._h, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(gw.data_ptr()), None)
    assert st == 4
