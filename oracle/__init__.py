"""CPU oracle for brute-force dedispersion -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this module. The product library never calls it and shares no
code with it (see dd_oracle.c for the arithmetic and its citations).

This wrapper marshals numpy arrays into the C routines of dd_oracle.c, which
are compiled with gcc on first use (or by `build()`). Inputs of every dtype
are decoded to float64 here (float16 by numpy, bfloat16 by placing the 16
stored bits above 16 zero bits of an IEEE float32), since the oracle sums the
values the device actually receives.

Parity status: every function here is pinned by tests/test_oracle_pins.py
against closed forms, special cases, hand-worked fixtures and brute force.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile dd_oracle.c into a shared library (gcc, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        _lib.oracle_shift_table.argtypes = [i32, P, f64, f64, i32, P, P]
        _lib.oracle_shift_table.restype = i32
        _lib.oracle_forward_f64.argtypes = [i32, i32, i32, i64, i64, P, P, P, P, P]
        _lib.oracle_forward_u8.argtypes = [i32, i32, i32, i64, i64, P, P, P, P]
        _lib.oracle_forward_points_f64.argtypes = [i32, i64, P, i64, P, P, i64, P, P, P, P, P]
        _lib.oracle_adjoint_f64.argtypes = [i32, i32, i32, i64, i64, P, P, P, P]
        _lib.oracle_grad_w_f64.argtypes = [i32, i32, i32, i64, i64, P, P, P, P]
        _lib.oracle_adjoint_points_f64.argtypes = [i32, i32, i64, P, P, P, i64, P, P, P, P, P]
        _lib.oracle_grad_w_channels_f64.argtypes = [i32, i32, i32, i64, i64, P, P, P, i64, P, P, P]
        _lib.oracle_forward_points_u8.argtypes = [i32, i64, P, i64, P, P, i64, P, P, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def decode(x: np.ndarray, dtype: str) -> np.ndarray:
    """Values of a stored input as float64 (bf16 given as uint16 bits)."""
    if dtype == "bf16":
        return (np.asarray(x, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return np.asarray(x).astype(np.float64)


def shift_table(freqs, f_ref, t_samp, dms) -> np.ndarray:
    """Eq. 1 delays in samples, int64 [n_dm][n_chan]."""
    lib = _load()
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    dm = np.ascontiguousarray(dms, dtype=np.float64)
    out = np.empty((dm.size, f.size), dtype=np.int64)
    rc = lib.oracle_shift_table(f.size, _p(f), float(f_ref), float(t_samp), dm.size, _p(dm), _p(out))
    if rc == -1:
        raise ValueError("invalid shift-table arguments")
    if rc == -2:
        raise ValueError("negative delay: a channel lies above the reference frequency")
    return out


def forward(x: np.ndarray, w: np.ndarray, shifts: np.ndarray, n_out: int,
            dtype: str = "f32", with_absum: bool = False):
    """Algorithm 1 with weights in float64. x: [B][C][stride] stored input.
    Returns out [B][D][S] float64 (and sum_c |w*x| if asked)."""
    lib = _load()
    xd = np.ascontiguousarray(decode(x, dtype))
    B, C, stride = xd.shape
    sh = np.ascontiguousarray(shifts, dtype=np.int64)
    D = sh.shape[0]
    assert sh.shape[1] == C and int(sh.max()) + n_out <= stride
    wd = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty((B, D, n_out), dtype=np.float64)
    ab = np.empty_like(out) if with_absum else None
    lib.oracle_forward_f64(B, C, D, n_out, stride, _p(xd), _p(wd), _p(sh), _p(out),
                           _p(ab) if with_absum else None)
    return (out, ab) if with_absum else out


def forward_u8(x: np.ndarray, wq: np.ndarray, shifts: np.ndarray, n_out: int) -> np.ndarray:
    """Exact integer forward for 8-bit input and integer weights (int64)."""
    lib = _load()
    xu = np.ascontiguousarray(x, dtype=np.uint8)
    B, C, stride = xu.shape
    sh = np.ascontiguousarray(shifts, dtype=np.int64)
    D = sh.shape[0]
    assert sh.shape[1] == C and int(sh.max()) + n_out <= stride
    wq64 = np.ascontiguousarray(wq, dtype=np.int64)
    out = np.empty((B, D, n_out), dtype=np.int64)
    lib.oracle_forward_u8(B, C, D, n_out, stride, _p(xu), _p(wq64), _p(sh), _p(out))
    return out


def forward_points(x: np.ndarray, w: np.ndarray, shifts: np.ndarray, pb, pd, pt,
                   dtype: str = "f32"):
    """Forward at the points (pb[i], pd[i], pt[i]); returns (values, absums)."""
    lib = _load()
    xd = np.ascontiguousarray(decode(x, dtype))
    B, C, stride = xd.shape
    sh = np.ascontiguousarray(shifts, dtype=np.int64)
    wd = np.ascontiguousarray(w, dtype=np.float64)
    pb, pd, pt = (np.ascontiguousarray(a, dtype=np.int64) for a in (pb, pd, pt))
    out = np.empty(pb.size, dtype=np.float64)
    ab = np.empty_like(out)
    lib.oracle_forward_points_f64(C, stride, _p(xd), C * stride, _p(wd), _p(sh), pb.size,
                                  _p(pb), _p(pd), _p(pt), _p(out), _p(ab))
    return out, ab


def forward_points_u8(x: np.ndarray, wq: np.ndarray, shifts: np.ndarray, pb, pd, pt):
    """Exact int64 forward of 8-bit input at the points (pb[i], pd[i], pt[i])."""
    lib = _load()
    xu = np.ascontiguousarray(x, dtype=np.uint8)
    B, C, stride = xu.shape
    sh = np.ascontiguousarray(shifts, dtype=np.int64)
    wq64 = np.ascontiguousarray(wq, dtype=np.int64)
    pb, pd, pt = (np.ascontiguousarray(a, dtype=np.int64) for a in (pb, pd, pt))
    out = np.empty(pb.size, dtype=np.int64)
    lib.oracle_forward_points_u8(C, stride, _p(xu), C * stride, _p(wq64), _p(sh), pb.size,
                                 _p(pb), _p(pd), _p(pt), _p(out))
    return out


def adjoint(g: np.ndarray, w: np.ndarray, shifts: np.ndarray, stride: int) -> np.ndarray:
    """Transpose of the forward w.r.t. the input (scatter form), float64
    [B][C][stride]."""
    lib = _load()
    gd = np.ascontiguousarray(g, dtype=np.float64)
    B, D, S = gd.shape
    sh = np.ascontiguousarray(shifts, dtype=np.int64)
    C = sh.shape[1]
    wd = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty((B, C, stride), dtype=np.float64)
    lib.oracle_adjoint_f64(B, C, D, S, stride, _p(gd), _p(wd), _p(sh), _p(out))
    return out


def grad_w(g: np.ndarray, x: np.ndarray, shifts: np.ndarray, dtype: str = "f32") -> np.ndarray:
    """d<g, forward(x, w)>/dw, float64 [C]."""
    lib = _load()
    gd = np.ascontiguousarray(g, dtype=np.float64)
    xd = np.ascontiguousarray(decode(x, dtype))
    B, D, S = gd.shape
    _, C, stride = xd.shape
    sh = np.ascontiguousarray(shifts, dtype=np.int64)
    out = np.empty(C, dtype=np.float64)
    lib.oracle_grad_w_f64(B, C, D, S, stride, _p(gd), _p(xd), _p(sh), _p(out))
    return out


def adjoint_points(g: np.ndarray, w: np.ndarray, shifts: np.ndarray, pb, pc, ptau):
    """Adjoint at input points (pb[i], pc[i], ptau[i]); returns (values, absums)."""
    lib = _load()
    gd = np.ascontiguousarray(g, dtype=np.float64)
    B, D, S = gd.shape
    sh = np.ascontiguousarray(shifts, dtype=np.int64)
    C = sh.shape[1]
    wd = np.ascontiguousarray(w, dtype=np.float64)
    pb, pc, ptau = (np.ascontiguousarray(a, dtype=np.int64) for a in (pb, pc, ptau))
    out = np.empty(pb.size, dtype=np.float64)
    ab = np.empty_like(out)
    lib.oracle_adjoint_points_f64(C, D, S, _p(gd), _p(wd), _p(sh), pb.size, _p(pb), _p(pc),
                                  _p(ptau), _p(out), _p(ab))
    return out, ab


def grad_w_channels(g: np.ndarray, x: np.ndarray, shifts: np.ndarray, chans, dtype: str = "f32"):
    """grad_w for the listed channels only; returns (values, absums)."""
    lib = _load()
    gd = np.ascontiguousarray(g, dtype=np.float64)
    xd = np.ascontiguousarray(decode(x, dtype))
    B, D, S = gd.shape
    _, C, stride = xd.shape
    sh = np.ascontiguousarray(shifts, dtype=np.int64)
    ch = np.ascontiguousarray(chans, dtype=np.int64)
    out = np.empty(ch.size, dtype=np.float64)
    ab = np.empty_like(out)
    lib.oracle_grad_w_channels_f64(B, C, D, S, stride, _p(gd), _p(xd), _p(sh), ch.size, _p(ch),
                                   _p(out), _p(ab))
    return out, ab
