"""One training step of the F-Hash INR, composed from the oracle's parts (test infrastructure only).

encode (Section 3.2.4) -> MLP -> MSE -> analytic backward -> table gradient scatter -> Adam
(Section 5.1.3).  Parameters are held in float64; the loss returned is the one computed on the
forward pass, before the update.
"""
import numpy as np

from . import adam, encode, mlp
from .schedule import bases


class Model:
    """Dense float64 state: table [rows][F], MLP flat vector, Adam moments and step count."""

    def __init__(self, levels, F, dims, table, mlp_params):
        self.levels = [list(map(int, R)) for R in levels]
        self.bases, self.rows = bases(self.levels)
        self.F, self.dims = F, list(dims)
        self.table = np.array(table, np.float64).reshape(self.rows, F)
        self.mlp = np.array(mlp_params, np.float64)
        self.m_t = np.zeros_like(self.table)
        self.v_t = np.zeros_like(self.table)
        self.m_w = np.zeros_like(self.mlp)
        self.v_w = np.zeros_like(self.mlp)
        self.k = 0

    def forward(self, coords):
        enc = encode.encode(self.levels, self.bases, coords, self.table)
        return mlp.forward(self.mlp, self.dims, enc)[0]


def loss_and_grads(levels, level_bases, F, dims, table, mlp_params, coords, targets, layout="linear"):
    """Returns (loss, y, MLP gradient, (rows, table gradient for those rows))."""
    enc = encode.encode(levels, level_bases, coords, table, layout)
    y, a, z = mlp.forward(mlp_params, dims, enc)
    L, g_y = mlp.mse(y, targets)
    g_mlp, d_enc = mlp.backward(mlp_params, dims, a, z, g_y)
    rows, g_tab = encode.encode_backward(levels, level_bases, coords, d_enc, F, layout)
    return L, y, g_mlp, (rows, g_tab)


def train_step(model, coords, targets, lr=1e-2, b1=0.9, b2=0.99, eps=1e-8):
    """One full step on `model` (in place); returns the loss of the forward pass."""
    L, _, g_mlp, (rows, g_rows) = loss_and_grads(model.levels, model.bases, model.F, model.dims,
                                                 model.table, model.mlp, coords, targets)
    g_tab = np.zeros_like(model.table)
    g_tab[rows] = g_rows
    model.k += 1
    model.table, model.m_t, model.v_t = adam.step(model.table, g_tab, model.m_t, model.v_t, model.k, lr, b1, b2, eps)
    model.mlp, model.m_w, model.v_w = adam.step(model.mlp, g_mlp, model.m_w, model.v_w, model.k, lr, b1, b2, eps)
    return L
