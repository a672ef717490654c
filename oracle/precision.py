"""bf16 precision form of the forward pass (oracle; test infrastructure only).

The precision form stores embeddings and MLP weights in bf16 (rounded to nearest, ties to even,
from the float32 master values) and feeds bf16 inputs to every layer's matrix product, the scalar
output layer included, with accumulation in float32 on the GPU.  This module rounds exactly the same
quantities to bf16 and then computes in float64, so the remaining difference to the GPU is its
float32 accumulation (and, rarely, a value on a bf16 rounding boundary that float32 and float64
round to neighbouring bf16 values).  Biases stay float32, as on the GPU.

Pins (tests/test_oracle_precision.py): bf16_round equals torch's bf16 conversion; with every table
value, weight, bias and activation already a bf16 value the emulation equals the float64 MLP exactly;
hand-worked single-neuron cases on rounding ties fix each rounding point (table values, the
interpolated layer-1 input, each weight matrix, each hidden activation before the next layer) and
that biases are not rounded; grads_bf16 equals torch float64 autograd of the same forward with the
roundings passed straight through and the float32 master weights in the backward.
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


class _RoundedRows:
    """A lazy table (indexable by row arrays, like oracle.rng.InitTable) read through bf16_round."""

    def __init__(self, table):
        self.table = table

    def __getitem__(self, rows):
        return bf16_round(np.asarray(self.table[rows], np.float32))


def _bf16_table(table):
    if isinstance(table, np.ndarray):
        return bf16_round(np.asarray(table, np.float32))
    return _RoundedRows(table)


def forward_bf16(levels, level_bases, table, params, dims, coords, layout="linear"):
    """y [N] of the precision form: bf16 table values, quadrilinear interpolation (float64), then every
    layer on bf16 inputs and bf16 weights with float32 biases (ReLU after the hidden layers).  `table`
    is a dense [rows][F] array or a lazy row-indexable table."""
    enc = encode.encode(levels, level_bases, coords, _bf16_table(table), layout)
    layers = mlp.unpack(params, dims)
    x = enc
    for k, (W, b) in enumerate(layers[:-1]):
        x = np.maximum(bf16_round(x) @ bf16_round(W).T + b, 0.0)
    Wo, bo = layers[-1]
    return (bf16_round(x) @ bf16_round(Wo).T + bo)[:, 0]


def grads_bf16(levels, level_bases, table, params, dims, coords, targets, layout="linear"):
    """Loss and MLP gradient of one training step in the precision form: the forward of forward_bf16
    (activations kept as computed), the MSE, and the backward in float64 with the float32 master
    weights (the GPU's backward reads those, and forms the weight gradients from the stored
    activations and deltas).  Also returns the sum of |terms| of each gradient entry, and the gradient
    of the loss with respect to the encoding, d_enc [N][L*F], with the sum of |terms| of each entry
    (encode.encode_backward turns both into table gradients)."""
    enc = encode.encode(levels, level_bases, coords, _bf16_table(table), layout)
    layers = mlp.unpack(params, dims)
    acts, pre = [enc], []
    x = enc
    for W, b in layers[:-1]:
        z = bf16_round(x) @ bf16_round(W).T + b
        pre.append(z)
        x = np.maximum(z, 0.0)
        acts.append(x)
    Wo, bo = layers[-1]
    y = (bf16_round(x) @ bf16_round(Wo).T + bo)[:, 0]
    L, gy = mlp.mse(y, targets)
    g, d_enc = mlp.backward(params, dims, acts, pre + [None], gy)
    gabs, d_enc_abs = mlp.backward(np.abs(params), dims, [np.abs(a) for a in acts],
                                   [np.where(z > 0, 1.0, -1.0) for z in pre] + [None], np.abs(gy))
    return L, g, gabs, d_enc, d_enc_abs
