"""Seeded synthetic inputs for the decoder: frames, masks, flows, residuals.

This module holds no arithmetic of the decoding method. It only draws the
inputs a decoder receives (mask positions and values, backward flow fields,
block residual data) and the synthetic source frames they were drawn from.
Both the CPU oracle and the CUDA path consume exactly these arrays.
"""
from .synth import (  # noqa: F401
    Residual,
    CoefResidual,
    IFrame,
    PFrame,
    PFrameCoef,
    Gop,
    block_grid,
    make_residual,
    make_coef_residual,
    coef_frame_residuals,
    make_config1,
    make_gop,
    make_iframe_only,
    make_flow_sinusoids,
)
