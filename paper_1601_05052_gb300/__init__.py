"""GB300-native brute-force dedispersion (Sclocco et al., arXiv:1601.05052).

Thin Python binding over libdd.so (include/dd.h). Every step of the
computation runs in the library's CUDA kernels; this module only marshals
arguments: PyTorch provides device memory and streams. There is no CPU
fallback: using a plan without a CUDA device raises.

    plan = Plan.from_setup(setup)              # Eq. 1 delay table + staging tables
    out = plan.execute(x, w)                   # x: [B][C][stride] on the GPU
    out = dedisperse(plan, x, w)               # autograd-aware (FP32 plans)
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import DDError, DTYPES, Variant, TuneReport  # noqa: F401

__all__ = ["Plan", "Batch", "Stream", "dedisperse", "compute_shifts", "DDError", "variants"]

_TORCH_DT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16,
             "u8": torch.uint8}


def _lib_():
    return _lib.load()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def compute_shifts(freqs, f_ref, t_samp, dms) -> np.ndarray:
    """Eq. 1 delay table int32 [n_dm][n_chan] (host only, no GPU needed)."""
    lib = _lib_()
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    dm = np.ascontiguousarray(dms, dtype=np.float64)
    out = np.empty((dm.size, f.size), dtype=np.int32)
    _lib.check(lib.dd_compute_shifts(f.size, f.ctypes.data, float(f_ref), float(t_samp),
                                     dm.size, dm.ctypes.data, out.ctypes.data))
    return out


def variants():
    """All compiled forward variants, as dicts."""
    lib = _lib_()
    out = []
    for i in range(lib.dd_variant_count()):
        v = Variant()
        _lib.check(lib.dd_variant_get(i, ctypes.byref(v)))
        out.append(v.as_dict())
    return out


class Plan:
    """A dedispersion plan: shapes, delay table and device staging tables."""

    def __init__(self, freqs=None, f_ref=None, t_samp=None, dms=None, n_out=None, batch=1,
                 dtype="f32", shifts=None):
        lib = _lib_()
        self.dtype = dtype
        self.batch = int(batch)
        self.n_out = int(n_out)
        h = ctypes.c_void_p()
        if shifts is not None:
            sh = np.ascontiguousarray(shifts, dtype=np.int32)
            self.n_dm, self.n_chan = sh.shape
            _lib.check(lib.dd_plan_create_from_shifts(ctypes.byref(h), self.n_chan, self.n_dm,
                                                      sh.ctypes.data, self.n_out, self.batch,
                                                      DTYPES[dtype]))
        else:
            f = np.ascontiguousarray(freqs, dtype=np.float64)
            dm = np.ascontiguousarray(dms, dtype=np.float64)
            self.n_chan, self.n_dm = f.size, dm.size
            _lib.check(lib.dd_plan_create(ctypes.byref(h), f.size, f.ctypes.data, float(f_ref),
                                          float(t_samp), dm.size, dm.ctypes.data, self.n_out,
                                          self.batch, DTYPES[dtype]))
        self._h = h
        self.input_len = lib.dd_plan_input_len(h)
        self.input_stride = lib.dd_plan_input_stride(h)
        self.max_shift = lib.dd_plan_max_shift(h)

    @classmethod
    def from_setup(cls, setup, dtype=None, batch=None):
        return cls(setup.freqs(), setup.f_ref, setup.t_samp, setup.dms(), setup.n_out,
                   batch=setup.batch if batch is None else batch, dtype=dtype or setup.dtype)

    def close(self):
        if getattr(self, "_h", None):
            _lib_().dd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- shapes ---------------------------------------------------------------
    @property
    def in_shape(self):
        return (self.batch, self.n_chan, self.input_stride)

    @property
    def out_shape(self):
        return (self.batch, self.n_dm, self.n_out)

    @property
    def torch_dtype(self):
        return _TORCH_DT[self.dtype]

    @property
    def out_dtype(self):
        return torch.int32 if self.dtype == "u8" else torch.float32

    @property
    def w_dtype(self):
        return torch.int32 if self.dtype == "u8" else torch.float32

    def shifts(self) -> np.ndarray:
        out = np.empty((self.n_dm, self.n_chan), dtype=np.int32)
        _lib.check(_lib_().dd_plan_shifts(self._h, out.ctypes.data))
        return out

    # -- variants / tuning ----------------------------------------------------
    @property
    def variant(self):
        v = Variant()
        _lib.check(_lib_().dd_plan_get_variant(self._h, ctypes.byref(v)))
        return v.as_dict()

    @variant.setter
    def variant(self, d):
        v = Variant(**d) if isinstance(d, dict) else Variant(*d)
        _lib.check(_lib_().dd_plan_set_variant(self._h, ctypes.byref(v)))

    @property
    def launch_order(self):
        """'dm' (DM tiles fastest, the default) or 'time' (time tiles fastest)."""
        o = ctypes.c_int32()
        _lib.check(_lib_().dd_plan_get_launch_order(self._h, ctypes.byref(o)))
        return "time" if o.value == 1 else "dm"

    @launch_order.setter
    def launch_order(self, order):
        _lib.check(_lib_().dd_plan_set_launch_order(self._h, {"dm": 0, "time": 1}[order]))

    def tune(self, budget_ms=0):
        r = TuneReport()
        _lib.check(_lib_().dd_tune(self._h, int(budget_ms), ctypes.byref(r)))
        return r.as_dict()

    def tune_adjoint(self, budget_ms=0):
        """Tunes the kernel variant the adjoint's transposed gather runs."""
        r = TuneReport()
        _lib.check(_lib_().dd_tune_adjoint(self._h, int(budget_ms), ctypes.byref(r)))
        return r.as_dict()

    @property
    def adjoint_variant(self):
        """The kernel variant of the adjoint's transposed gather (FP32 plans)."""
        v = Variant()
        _lib.check(_lib_().dd_adjoint_get_variant(self._h, ctypes.byref(v)))
        return v.as_dict()

    @adjoint_variant.setter
    def adjoint_variant(self, d):
        v = Variant(**d) if isinstance(d, dict) else Variant(*d)
        _lib.check(_lib_().dd_adjoint_set_variant(self._h, ctypes.byref(v)))

    def check_device(self):
        _lib.check(_lib_().dd_plan_check_device(self._h))

    # -- compute --------------------------------------------------------------
    def _check_in(self, x, w):
        if not (x.is_cuda and w.is_cuda):
            raise ValueError("inputs must be CUDA tensors (no CPU path)")
        if w.device != x.device:
            raise ValueError("input and weights must be on one device")
        if tuple(x.shape) != self.in_shape or x.dtype != self.torch_dtype or not x.is_contiguous():
            raise ValueError("input must be contiguous %s %s, got %s %s"
                             % (self.in_shape, self.torch_dtype, tuple(x.shape), x.dtype))
        if tuple(w.shape) != (self.n_chan,) or w.dtype != self.w_dtype or not w.is_contiguous():
            raise ValueError("weights must be contiguous [%d] %s" % (self.n_chan, self.w_dtype))

    @staticmethod
    def _check_buf(t, shape, dtype, device, what):
        """A caller-supplied device buffer: its pointer goes to a kernel as is,
        so it must be a contiguous CUDA tensor of the exact shape and type on
        the input's device."""
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device != device:
            raise ValueError("%s must be a CUDA tensor on %s" % (what, device))
        if tuple(t.shape) != tuple(shape) or t.dtype != dtype or not t.is_contiguous():
            raise ValueError("%s must be contiguous %s %s, got %s %s"
                             % (what, tuple(shape), dtype, tuple(t.shape), t.dtype))

    def empty_input(self, device="cuda"):
        return torch.empty(self.in_shape, dtype=self.torch_dtype, device=device)

    def execute(self, x, w, out=None, stream=None):
        """Forward on the current (or given) stream; returns `out`."""
        self._check_in(x, w)
        if out is None:
            out = torch.empty(self.out_shape, dtype=self.out_dtype, device=x.device)
        else:
            self._check_buf(out, self.out_shape, self.out_dtype, x.device, "out")
        _lib.check(_lib_().dd_execute(self._h, _ptr(x), _ptr(w), _ptr(out), _stream(stream)))
        return out

    def execute_host(self, x, w, out, stream=None):
        """Forward from/to host tensors (pinned for full speed); synchronous.
        The library reads and writes whole buffers of the plan's shapes
        through these pointers (over the CPU-GPU link when pinned), so each
        must be a contiguous host tensor of exactly that shape and type."""
        for t, shape, dtype, what in ((x, self.in_shape, self.torch_dtype, "x"),
                                      (w, (self.n_chan,), self.w_dtype, "w"),
                                      (out, self.out_shape, self.out_dtype, "out")):
            if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous():
                raise ValueError("execute_host takes contiguous host tensors (%s)" % what)
            if tuple(t.shape) != tuple(shape) or t.dtype != dtype:
                raise ValueError("%s must be %s %s, got %s %s"
                                 % (what, tuple(shape), dtype, tuple(t.shape), t.dtype))
        _lib.check(_lib_().dd_execute_host(self._h, _ptr(x), _ptr(w), _ptr(out),
                                           _stream(stream)))
        return out

    def adjoint(self, g, w=None, x=None, need_gin=True, need_gw=True, stream=None):
        """(grad_in [B][C][stride] or None, grad_w [C] or None) for cotangent g."""
        if self.dtype != "f32":
            raise ValueError("the adjoint takes FP32 plans only")
        g = g.contiguous()
        if tuple(g.shape) != self.out_shape or g.dtype != torch.float32 or not g.is_cuda:
            raise ValueError("cotangent must be CUDA float32 %s" % (self.out_shape,))
        if need_gin:
            if w is None:
                raise ValueError("the input gradient needs the weights")
            self._check_buf(w, (self.n_chan,), torch.float32, g.device, "w")
        if need_gw:
            if x is None:
                raise ValueError("the weight gradient needs the input")
            self._check_buf(x, self.in_shape, torch.float32, g.device, "x")
        gin = torch.empty(self.in_shape, dtype=torch.float32, device=g.device) if need_gin else None
        gw = torch.empty(self.n_chan, dtype=torch.float32, device=g.device) if need_gw else None
        _lib.check(_lib_().dd_adjoint(self._h, _ptr(g), _ptr(w), _ptr(x), _ptr(gin), _ptr(gw),
                                      _stream(stream)))
        return gin, gw


class _Dedisperse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, plan):
        ctx.plan = plan
        ctx.save_for_backward(x, w)
        return plan.execute(x, w)

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        gin, gw = ctx.plan.adjoint(g, w, x, need_gin=ctx.needs_input_grad[0],
                                   need_gw=ctx.needs_input_grad[1])
        return gin, gw, None


def dedisperse(plan, x, w):
    """Autograd-aware forward: d/dx and d/dw come from the adjoint kernels."""
    return _Dedisperse.apply(x, w, plan)


class Batch:
    """Several plans run by one persistent, graph-replayed kernel launch."""

    def __init__(self, plans):
        lib = _lib_()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _lib.check(lib.dd_batch_create(ctypes.byref(h), len(self.plans), arr))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib_().dd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def variant(self):
        v = Variant()
        _lib.check(_lib_().dd_batch_get_variant(self._h, ctypes.byref(v)))
        return v.as_dict()

    @variant.setter
    def variant(self, d):
        v = Variant(**d) if isinstance(d, dict) else Variant(*d)
        _lib.check(_lib_().dd_batch_set_variant(self._h, ctypes.byref(v)))

    def plan_variant(self, i):
        """The variant plan i runs in this batch (its own tile split and chunk)."""
        v = Variant()
        _lib.check(_lib_().dd_batch_get_plan_variant(self._h, int(i), ctypes.byref(v)))
        return v.as_dict()

    def set_plan_variant(self, i, d):
        v = Variant(**d) if isinstance(d, dict) else Variant(*d)
        _lib.check(_lib_().dd_batch_set_plan_variant(self._h, int(i), ctypes.byref(v)))

    @property
    def plan_variants(self):
        return [self.plan_variant(i) for i in range(len(self.plans))]

    def tune(self, budget_ms=0):
        r = TuneReport()
        _lib.check(_lib_().dd_batch_tune(self._h, int(budget_ms), ctypes.byref(r)))
        return r.as_dict()

    def execute(self, xs, ws, outs=None, stream=None):
        n = len(self.plans)
        if len(xs) != n or len(ws) != n or (outs is not None and len(outs) != n):
            raise ValueError("one input, weight vector and output per plan (%d)" % n)
        for p, x, w in zip(self.plans, xs, ws):
            p._check_in(x, w)
        if outs is None:
            outs = [torch.empty(p.out_shape, dtype=p.out_dtype, device=x.device)
                    for p, x in zip(self.plans, xs)]
        else:
            for i, (p, x, o) in enumerate(zip(self.plans, xs, outs)):
                Plan._check_buf(o, p.out_shape, p.out_dtype, x.device, "outs[%d]" % i)
        A = ctypes.c_void_p * n
        _lib.check(_lib_().dd_batch_execute(
            self._h, A(*[x.data_ptr() for x in xs]), A(*[w.data_ptr() for w in ws]),
            A(*[o.data_ptr() for o in outs]), _stream(stream)))
        return outs


class Stream:
    """Continuous dedispersion in chunks of `plan.n_out` samples per channel.

    push(chunk [B][C][n_out]) returns the output samples
    [k*n_out - latency, (k+1)*n_out - latency) of the continuous stream."""

    def __init__(self, plan):
        self.plan = plan
        h = ctypes.c_void_p()
        _lib.check(_lib_().dd_stream_create(ctypes.byref(h), plan._h))
        self._h = h
        self.latency = _lib_().dd_stream_latency(h)

    def close(self):
        if getattr(self, "_h", None):
            _lib_().dd_stream_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        _lib.check(_lib_().dd_stream_reset(self._h, _stream(stream)))

    def push(self, chunk, w, out=None, stream=None):
        p = self.plan
        shape = (p.batch, p.n_chan, p.n_out)
        if (tuple(chunk.shape) != shape or chunk.dtype != p.torch_dtype or not chunk.is_cuda
                or not chunk.is_contiguous()):
            raise ValueError("chunk must be a contiguous CUDA %s %s" % (shape, p.torch_dtype))
        p._check_buf(w, (p.n_chan,), p.w_dtype, chunk.device, "weights")
        if out is None:
            out = torch.empty(p.out_shape, dtype=p.out_dtype, device=chunk.device)
        else:
            p._check_buf(out, p.out_shape, p.out_dtype, chunk.device, "out")
        _lib.check(_lib_().dd_stream_push(self._h, _ptr(chunk), _ptr(w), _ptr(out),
                                          _stream(stream)))
        return out
