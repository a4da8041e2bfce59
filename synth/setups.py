"""Observation setups used as synthetic stand-ins for the paper's workloads.

The paper's two setups (Section IV): "Apertif" (20 000 samples/s, 1024
channels of 300/1024 MHz from 1420 MHz, DM step 0.25) and "LOFAR" (200 000
samples/s, 32 channels of ~0.19 MHz from 138 MHz, DM step 0.25), both
starting at DM 0. The benchmark workloads below use the same conventions.

Channel frequencies follow the band-edge convention: with C channels over
[lo, hi), channel c sits at f_c = lo + c * (hi - lo) / C, ascending in memory,
and the reference frequency is the top channel, f_ref = hi - (hi - lo) / C.
"""
from dataclasses import dataclass, field
import numpy as np


@dataclass(frozen=True)
class Setup:
    name: str
    n_chan: int
    f_lo: float          # MHz, lower band edge (= frequency of channel 0)
    f_hi: float          # MHz, upper band edge
    t_samp: float        # seconds
    dm0: float           # first trial DM, pc/cm^3
    ddm: float           # DM step
    n_dm: int
    n_out: int           # output samples per DM trial (S)
    batch: int = 1       # beams
    dtype: str = "f32"   # input dtype: f32 | f16 | bf16 | u8
    note: str = ""

    @property
    def chan_width(self) -> float:
        return (self.f_hi - self.f_lo) / self.n_chan

    def freqs(self) -> np.ndarray:
        return self.f_lo + np.arange(self.n_chan, dtype=np.float64) * self.chan_width

    @property
    def f_ref(self) -> float:
        return self.f_hi - self.chan_width

    def dms(self) -> np.ndarray:
        return self.dm0 + np.arange(self.n_dm, dtype=np.float64) * self.ddm

    def with_(self, **kw) -> "Setup":
        d = dict(self.__dict__)
        d.update(kw)
        return Setup(**d)


SETUPS = {
    # plain FP32, one beam, 64 channels over 1400-1500 MHz, 64 us, DMs 0..31.5.
    "lband64": Setup("lband64", 64, 1400.0, 1500.0, 64e-6, 0.0, 0.5, 64, 4096),
    # survey scale, Apertif-like: 1024 ch over 1420-1720 MHz, 50 us, 2048 DMs step 0.25.
    "apertif_survey": Setup("apertif_survey", 1024, 1420.0, 1720.0, 50e-6, 0.0, 0.25, 2048, 20000),
    # the precision forms of lband64 (u8 / f16 / bf16 inputs, weighted).
    "lband64_u8": Setup("lband64_u8", 64, 1400.0, 1500.0, 64e-6, 0.0, 0.5, 64, 4096, dtype="u8"),
    "lband64_f16": Setup("lband64_f16", 64, 1400.0, 1500.0, 64e-6, 0.0, 0.5, 64, 4096, dtype="f16"),
    "lband64_bf16": Setup("lband64_bf16", 64, 1400.0, 1500.0, 64e-6, 0.0, 0.5, 64, 4096, dtype="bf16"),
    # batched uneven beams: 96 beams of the lband64 shape plus 32 low-frequency beams
    # (256 ch over 120-180 MHz, 204.8 us, 2000 DMs step 0.05).
    "lband64_x96_u8": Setup("lband64_x96_u8", 64, 1400.0, 1500.0, 64e-6, 0.0, 0.5, 64, 4096, batch=96, dtype="u8"),
    "lowfreq256_u8": Setup("lowfreq256_u8", 256, 120.0, 180.0, 204.8e-6, 0.0, 0.05, 2000, 10000, batch=32, dtype="u8"),
    # differentiable weighted dedispersion, 16 beams of 512 ch over 1250-1550 MHz.
    "diff16_512ch": Setup("diff16_512ch", 512, 1250.0, 1550.0, 100e-6, 0.0, 0.25, 1024, 8192, batch=16),
    # extra measurement point: the lband64 shape at 96 beams in FP32 (leaves L2).
    "lband64_x96": Setup("lband64_x96", 64, 1400.0, 1500.0, 64e-6, 0.0, 0.5, 64, 4096, batch=96),
    # an HBM-bound point: the lband64 band with only 4 trial DMs (0-1.5) over 384 beams
    # (~0.6 adds per compulsory byte, far below the FP32 ridge).
    "lband64_4dm_x384": Setup("lband64_4dm_x384", 64, 1400.0, 1500.0, 64e-6, 0.0, 0.5, 4, 4096,
                              batch=384),
    # the paper's LOFAR-like setup (32 ch x 0.1953125 MHz from 138 MHz, 5 us).
    "lofar": Setup("lofar", 32, 138.0, 138.0 + 32 * 0.1953125, 5e-6, 0.0, 0.25, 2048, 200000),
    # Apertif DM = 0 "perfect reuse" form (all trial DMs zero).
    "apertif_survey_dm0": Setup("apertif_survey_dm0", 1024, 1420.0, 1720.0, 50e-6, 0.0, 0.0, 2048, 20000),
}


def setup(name: str) -> Setup:
    return SETUPS[name]
