"""bf16 precision form of the forward pass (oracle; test infrastructure only).

The precision form stores embeddings and MLP weights in bf16 (rounded to nearest, ties to even,
from the float32 master values) and feeds bf16 inputs to each hidden layer's matrix product, with
accumulation in float32 on the GPU.  This module rounds exactly the same quantities to bf16 and then
computes in float64, so the remaining difference to the GPU is its float32 accumulation (and, rarely,
a value on a bf16 rounding boundary that float32 and float64 round to neighbouring bf16 values).
Biases and the scalar output layer stay float32, as on the GPU.
"""
import numpy as np

from . import encode, mlp


def bf16_round(x):
    """Round float values to the nearest bf16 (ties to even), returned as float64 (NaN preserved)."""
    f = np.asarray(x, np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    rounded = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


def forward_bf16(levels, level_bases, table, params, dims, coords):
    """y [N] of the precision form: bf16 table values, quadrilinear interpolation (float64), then each
    hidden layer on bf16 inputs and bf16 weights, float32 biases; output layer on unrounded inputs."""
    enc = encode.encode(levels, level_bases, coords, bf16_round(np.asarray(table, np.float32)))
    layers = mlp.unpack(params, dims)
    x = enc
    for k, (W, b) in enumerate(layers[:-1]):
        x = np.maximum(bf16_round(x) @ bf16_round(W).T + b, 0.0)
    Wo, bo = layers[-1]
    return (x @ Wo.T + bo)[:, 0]
