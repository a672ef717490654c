"""Shallow MLP decoder, MSE loss and analytic backward (oracle; test infrastructure only).

Section 3.2.4 feeds the concatenated level encodings to a shallow MLP; Section 4.2 fixes
2 hidden layers of 64 neurons for the experiments.  The activation is not stated: the reading
is ReLU on hidden layers, a linear scalar output and a bias on every layer (PyTorch
nn.Linear), with ReLU'(0) = 0.  Training minimises the mean squared error.

Flat parameter layout, layer by layer: W[out][in] (row-major) then b[out].
"""
import numpy as np


def unpack(params, dims):
    """Split the flat vector into [(W, b), ...] float64 views."""
    p = np.asarray(params, np.float64)
    out, o = [], 0
    for k in range(len(dims) - 1):
        fi, fo = dims[k], dims[k + 1]
        W = p[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = p[o:o + fo]
        o += fo
        out.append((W, b))
    return out


def n_params(dims):
    return sum(dims[k] * dims[k + 1] + dims[k + 1] for k in range(len(dims) - 1))


def forward(params, dims, x):
    """Returns (y [N], activations list a_0..a_{K-1}, pre-activations list z_1..z_K)."""
    layers = unpack(params, dims)
    a = [np.asarray(x, np.float64)]
    z = []
    for k, (W, b) in enumerate(layers):
        zk = a[-1] @ W.T + b
        z.append(zk)
        if k < len(layers) - 1:
            a.append(np.maximum(zk, 0.0))
    return z[-1][:, 0], a, z


def mse(y, target):
    """Mean squared error and its gradient with respect to y."""
    r = np.asarray(y, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(r * r)), 2.0 * r / r.size


def backward(params, dims, a, z, g_y):
    """Analytic backward of forward(): returns (flat parameter gradient, d_input [N][dims[0]])."""
    layers = unpack(params, dims)
    g = np.asarray(g_y, np.float64)[:, None]
    grads = [None] * len(layers)
    for k in range(len(layers) - 1, -1, -1):
        W, _ = layers[k]
        grads[k] = (g.T @ a[k], g.sum(axis=0))
        g = g @ W
        if k > 0:
            g = g * (z[k - 1] > 0.0)
    flat = np.concatenate([np.concatenate([dW.reshape(-1), db]) for dW, db in grads])
    return flat, g
