"""The float32 MLP of the training step on the tensor cores against the oracle (GPU, through the C ABI).

fhash_compute_grads runs the MLP's forward, loss and backward data path as one fused tensor-core
kernel (3xTF32 GEMMs) whenever the shape allows it: encoding width 16, 32 or 64, hidden width 64, one
or two hidden layers.  Every such shape is checked here at batch sizes below one 128-sample tile,
ragged (not a multiple of the tile) and spanning more tiles than the GPU has SMs (each CTA then walks
several tiles).  The loss must match to 1e-5 relative, and every MLP and table gradient entry must be
within 1e-4 of the sum of the magnitudes of its terms.  These are the bounds of the SIMT path's test.
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import encode, mlp, train

from _util import fh, read, set_params, to_dev

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


def _res(L):
    """L levels, geometric from 4^3 x 1 to 32^3 x 8 (rounded)."""
    return [[int(round(4 * 8 ** (l / (L - 1))))] * 3 + [int(round(8 ** (l / (L - 1))))] for l in range(L)]


@pytest.fixture(scope="module")
def field_mask():
    return workloads.make_field_and_mask(W1)


@pytest.mark.parametrize("L,F,hidden,n", [(8, 2, 2, 3000), (16, 2, 2, 70001), (16, 4, 1, 5000), (8, 8, 2, 100),
                                          (16, 1, 1, 4097)])
def test_tc_mlp_gradients(field_mask, L, F, hidden, n):
    f, m = field_mask
    nx, ny, nz, nt = W1["dims"]
    model = fh().fhash_build(nx, ny, nz, nt, mask=m, schedule=fh().make_schedule(mode="explicit", res=_res(L)), F=F,
                             mlp_hidden_layers=hidden, mlp_width=64, seed=9, init_range=0.5)
    info = fh().fhash_get_info(model)
    assert info["mlp_dims"] == [L * F] + [64] * hidden + [1]
    table = synth.uniform(31, 50, info["n_table_params"], -0.5, 0.5)
    p = synth.init_mlp(31, info["mlp_dims"])
    set_params(model, table, p)
    c = synth.coords(17, n)
    tgt = synth.sample(f, info["fbb_lo"], info["fbb_size"], c)
    loss = np.zeros(1, np.float64)
    fh().fhash_compute_grads(model, to_dev(c), to_dev(tgt), loss)
    T = table.reshape(-1, F).astype(np.float64)
    Lo, _, g_mlp, (rows, g_rows) = train.loss_and_grads(info["res"], info["base"], F, info["mlp_dims"], T, p, c, tgt)
    assert abs(loss[0] - Lo) <= 1e-5 * Lo
    n_t = info["n_table_params"]
    g = read(model, fh().STATE_GRAD, 0, n_t + info["n_mlp_params"])
    enc = encode.encode(info["res"], info["base"], c, T)
    y, a, z = mlp.forward(p, info["mlp_dims"], enc)
    _, gy = mlp.mse(y, tgt)
    abs_mlp, abs_denc = mlp.backward(np.abs(p), info["mlp_dims"], [np.abs(x) for x in a],
                                     [np.where(x > 0, 1.0, -1.0) for x in z], np.abs(gy))
    assert (np.abs(g[n_t:] - g_mlp) <= 1e-4 * abs_mlp + 1e-12).all()
    _, g_abs = encode.encode_backward(info["res"], info["base"], c, abs_denc, F)
    gt = g[:n_t].reshape(-1, F)
    assert (np.abs(gt[rows] - g_rows) <= 1e-4 * g_abs + 1e-12).all()
    untouched = np.ones(gt.shape[0], bool)
    untouched[rows] = False
    assert (gt[untouched] == 0).all()
