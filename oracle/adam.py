"""Adam (Section 5.1.3: Adam, initial learning rate 0.01), PyTorch semantics, float64.

Dense update of every parameter at every step (PyTorch's default for dense tensors, so rows a
batch does not touch still move through their first moment), bias-corrected, no weight decay:
  m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
  p <- p - lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps),   k = 1, 2, ...
Oracle; test infrastructure only.
"""
import numpy as np


def step(p, g, m, v, k, lr=1e-2, b1=0.9, b2=0.99, eps=1e-8):
    """One Adam step at step count k (1-based).  Returns new (p, m, v) as float64 arrays."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** k)
    vhat = v / (1.0 - b2 ** k)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
