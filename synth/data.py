"""Seeded synthetic data: Gaussian noise, dispersed pulses, channel weights.

Recipe (all draws from numpy's PCG64 `default_rng(seed)`):

* noise: i.i.d. N(0, 1) float32, shape [batch][n_chan][T_in];
* pulses: each pulse (beam b, trial index d*, time t0, amplitude A) adds A to
  in[b][c][t0 + shift[d*][c]] for every channel c, after the noise, so that it
  lines up exactly at trial d*; the shift table is supplied by the caller;
* uint8 input: clip(round(128 + 16 * x), 0, 255) of the float32 noise+pulses x
  (mean 128, sd 16, halves rounded to even);
* float16 input: x cast to float16 (round to nearest even);
* bfloat16 input: x rounded to nearest even bfloat16, kept as uint16 bit
  patterns (numpy has no bfloat16 type);
* weights: ones, or U(0.5, 1.5) with round(5% * C) channels zeroed by a seeded
  permutation (RFI-masked channels). Integer weights for 8-bit input are the
  Q8 values round(256 * w).

Rows are padded to a stride that is a multiple of 16 bytes; pad entries hold
`pad_value` (NaN by default for float types, so any use of them shows up).
"""
import numpy as np

ELT_BYTES = {"f32": 4, "f16": 2, "bf16": 2, "u8": 1}


def padded_stride(t_in: int, dtype: str) -> int:
    """Smallest row length >= t_in whose size in bytes is a multiple of 16."""
    q = 16 // ELT_BYTES[dtype]
    return ((t_in + q - 1) // q) * q


def to_f16(x: np.ndarray) -> np.ndarray:
    return x.astype(np.float16)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns, round to nearest, ties to even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)
    nan = np.isnan(x)
    if nan.any():
        r[nan] = 0x7FC0
    return r


def bf16_bits_to_f32(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


def quantize_u8(x: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(128.0 + 16.0 * x.astype(np.float64)), 0, 255).astype(np.uint8)


def pulse_plan(setup, seed: int, n_per_beam: int = 1, amp=(3.0, 10.0),
               fixed=None):
    """List of (beam, trial index, t0, amplitude). `fixed` = (d, t0, A) puts
    the same pulse in every beam (the 1-beam workloads fix DM 20.0 at t=1000,
    A=5); otherwise indices, times and amplitudes are drawn from the seed."""
    rng = np.random.default_rng(seed + 1_000_003)
    out = []
    for b in range(setup.batch):
        for _ in range(n_per_beam):
            if fixed is not None:
                out.append((b, int(fixed[0]), int(fixed[1]), float(fixed[2])))
            else:
                d = int(rng.integers(0, setup.n_dm))
                t0 = int(rng.integers(0, setup.n_out))
                a = float(rng.uniform(amp[0], amp[1]))
                out.append((b, d, t0, a))
    return out


def make_input(setup, shifts: np.ndarray, seed: int, dtype: str = None,
               pulses=None, pad_value=None, t_in: int = None):
    """Seeded input [batch][n_chan][stride] in `dtype` (bf16 as uint16 bits).

    shifts: int [n_dm][n_chan] table from the side under test (only used to
    place pulses and to size T_in = n_out + max shift)."""
    dtype = dtype or setup.dtype
    B, C, S = setup.batch, setup.n_chan, setup.n_out
    shifts = np.asarray(shifts)
    if t_in is None:
        t_in = S + int(shifts.max())
    stride = padded_stride(t_in, dtype)
    rng = np.random.default_rng(seed)
    np_dt = {"f32": np.float32, "f16": np.float16, "bf16": np.uint16, "u8": np.uint8}[dtype]
    out = np.empty((B, C, stride), dtype=np_dt)
    if pad_value is None:
        pad_value = {"f32": np.float32(np.nan), "f16": np.float16(np.nan),
                     "bf16": np.uint16(0x7FC0), "u8": np.uint8(0xA5)}[dtype]
    out[:, :, t_in:] = pad_value
    by_beam = {}
    for (b, d, t0, a) in (pulses or []):
        by_beam.setdefault(b, []).append((d, t0, a))
    cidx = np.arange(C)
    for b in range(B):
        x = rng.standard_normal((C, t_in), dtype=np.float32)
        for (d, t0, a) in by_beam.get(b, []):
            x[cidx, t0 + shifts[d]] += np.float32(a)
        if dtype == "f32":
            out[b, :, :t_in] = x
        elif dtype == "f16":
            out[b, :, :t_in] = to_f16(x)
        elif dtype == "bf16":
            out[b, :, :t_in] = to_bf16_bits(x)
        else:
            out[b, :, :t_in] = quantize_u8(x)
    return out


def make_weights(n_chan: int, seed: int, kind: str = "ones", masked_frac: float = 0.05):
    """Per-channel float32 weights: 'ones', or 'uniform' = U(0.5, 1.5) with
    round(masked_frac * n_chan) channels set to 0 by a seeded permutation."""
    if kind == "ones":
        return np.ones(n_chan, dtype=np.float32)
    rng = np.random.default_rng(seed + 7_000_001)
    w = rng.uniform(0.5, 1.5, size=n_chan).astype(np.float32)
    n_mask = int(round(masked_frac * n_chan))
    w[rng.permutation(n_chan)[:n_mask]] = 0.0
    return w


def quantize_weights_q8(w: np.ndarray) -> np.ndarray:
    """Integer weights for 8-bit input: round(256 * w), halves up."""
    return np.floor(256.0 * w.astype(np.float64) + 0.5).astype(np.int32)
