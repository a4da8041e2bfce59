"""Seeded synthetic workloads for dedispersion.

This package only *describes and draws* inputs: observation setups (channel
frequencies, trial-DM lists, sample counts) and seeded noise, pulses and
weights. It holds none of the method's arithmetic: wherever a dispersed pulse
has to be placed, the caller passes in a shift table computed by whichever
side (oracle or library) is under test. Both the oracle-based tests and the
CUDA path draw their inputs from here, so the two see identical data.
"""
from .setups import Setup, SETUPS, setup  # noqa: F401
from .data import (  # noqa: F401
    padded_stride, make_input, quantize_u8, to_f16, to_bf16_bits, bf16_bits_to_f32,
    make_weights, quantize_weights_q8, pulse_plan,
)
