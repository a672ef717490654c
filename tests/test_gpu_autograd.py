"""The encoding's backward (fhash_encode_backward) and its torch.autograd wrapper, against the oracle.

- fhash_encode_backward on 5000 ragged samples with d(encoding) drawn at random: every table gradient
  within 1e-5 x the sum of the magnitudes of its terms; untouched rows exactly zero; a second call
  accumulates (twice the first).
- Central finite differences of L(T) = sum(R * encode(T)) through fhash_encode alone, on 48 table
  elements touched at the coarsest, a middle and the finest level (L is linear in T, so the
  difference quotient is exact up to float32 rounding of the encoding).
- A torch MLP on top of the autograd Encoding module: loss.backward() gives table gradients equal to
  the oracle's analytic ones (Eqs. 10-12 backward after the MLP backward) within 1e-4 x the sum of
  term magnitudes, and torch's MLP gradients equal the oracle's.
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import encode, mlp, train

from _util import build, fh, read, set_params, to_dev, torch

pytestmark = pytest.mark.gpu
W = workloads.SMALL


@pytest.fixture()
def small():
    f, m = workloads.make_field_and_mask(W)
    model = build(W, mask=m)
    info = fh().fhash_get_info(model)
    table = synth.uniform(5, 50, info["n_table_params"], -1.0, 1.0)
    p = synth.init_mlp(5, info["mlp_dims"])
    set_params(model, table, p)
    return dict(field=f, model=model, info=info, table=table.reshape(-1, info["F"]), mlp=p)


def _table_grad(model, info):
    return read(model, fh().STATE_GRAD, 0, info["n_table_params"]).reshape(-1, info["F"]).astype(np.float64)


def test_encode_backward_matches_oracle(small):
    info, model = small["info"], small["model"]
    lv, b, F, L = info["res"], info["base"], info["F"], info["n_levels"]
    n = 5000
    c = synth.coords(21, n)
    d = synth.uniform(22, 60, n * L * F, -1.0, 1.0).reshape(n, L * F)
    dc, dd = to_dev(c), to_dev(d)
    fh().fhash_encode_backward(model, dc, dd)
    got = _table_grad(model, info)

    rows, g = encode.encode_backward(lv, b, c, d, F)
    _, g_abs = encode.encode_backward(lv, b, c, np.abs(d), F)
    ref = np.zeros_like(got)
    ref[rows] = g
    bound = np.zeros_like(got)
    bound[rows] = g_abs
    assert (np.abs(got - ref) <= 1e-5 * bound + 1e-30).all()
    untouched = np.ones(got.shape[0], bool)
    untouched[rows] = False
    assert (got[untouched] == 0).all()

    fh().fhash_encode_backward(model, dc, dd)  # accumulates
    got2 = _table_grad(model, info)
    assert (np.abs(got2 - 2 * ref) <= 2e-5 * bound + 1e-30).all()

    fh().fhash_encode_backward(model, dc[:0], dd[:0])  # n = 0: no-op
    with pytest.raises(fh().FHashError):
        fh().fhash_encode_backward(model, c, d)  # host buffers are rejected


def test_encode_backward_finite_differences(small):
    info, model = small["info"], small["model"]
    lv, b, F, L = info["res"], info["base"], info["F"], info["n_levels"]
    n = 3000
    c = synth.coords(23, n)
    R = synth.uniform(24, 61, n * L * F, -1.0, 1.0).reshape(n, L * F).astype(np.float64)
    dc = to_dev(c)
    fh().fhash_encode_backward(model, dc, to_dev(R.astype(np.float32)))
    g = _table_grad(model, info)
    enc = torch().empty((n, L * F), dtype=torch().float32, device="cuda")

    def loss():
        fh().fhash_encode(model, dc, enc)
        return float((enc.cpu().numpy().astype(np.float64) * R).sum())

    pick = np.random.default_rng(4)
    h = 5e-2
    checked = 0
    for level in (0, L // 2, L - 1):
        rows, _ = encode.level_corners(c, lv[level], b[level])
        for r in pick.choice(np.unique(rows), 16, replace=False):
            f = int(pick.integers(0, F))
            off = int(r) * F + f
            v0 = small["table"][r, f]
            fh().fhash_write_state(model, fh().STATE_PARAM, off, np.array([v0 + h], np.float32))
            lp = loss()
            fh().fhash_write_state(model, fh().STATE_PARAM, off, np.array([v0 - h], np.float32))
            lm = loss()
            fh().fhash_write_state(model, fh().STATE_PARAM, off, np.array([v0], np.float32))
            hh = (np.float64(np.float32(v0 + h)) - np.float64(np.float32(v0 - h))) / 2
            fd = (lp - lm) / (2 * hh)
            assert abs(fd - g[r, f]) <= 1e-3 * abs(g[r, f]) + 2e-4, (level, r, f, fd, g[r, f])
            checked += 1
    assert checked == 48


def test_autograd_encoding_with_torch_mlp(small):
    t = torch()
    from paper_2507_03836_gb300.autograd import Encoding
    info, model = small["info"], small["model"]
    lv, b, F, dims = info["res"], info["base"], info["F"], info["mlp_dims"]
    n = 4097
    c = synth.coords(25, n)
    tgt = synth.sample(small["field"], info["fbb_lo"], info["fbb_size"], c)

    layers, off = [], 0
    for k in range(len(dims) - 1):
        fi, fo = dims[k], dims[k + 1]
        lin = t.nn.Linear(fi, fo).cuda()
        with t.no_grad():
            lin.weight.copy_(t.from_numpy(small["mlp"][off:off + fo * fi].reshape(fo, fi)))
            lin.bias.copy_(t.from_numpy(small["mlp"][off + fo * fi:off + fo * fi + fo]))
        off += fo * fi + fo
        layers += [lin, t.nn.ReLU()] if k < len(dims) - 2 else [lin]
    net = t.nn.Sequential(*layers)
    prev = t.backends.cuda.matmul.allow_tf32
    t.backends.cuda.matmul.allow_tf32 = False
    try:
        encoder = Encoding(model)
        y = net(encoder(to_dev(c)))[:, 0]
        loss = ((y - to_dev(tgt)) ** 2).mean()
        loss.backward()
        t.cuda.synchronize()
    finally:
        t.backends.cuda.matmul.allow_tf32 = prev

    Lref, _, g_mlp, (rows, g_rows) = train.loss_and_grads(lv, b, F, dims, small["table"], small["mlp"], c, tgt)
    assert abs(float(loss.detach()) - Lref) <= 1e-5 * Lref
    # term-magnitude bound of the table gradient
    enc = encode.encode(lv, b, c, small["table"])
    yy, a, z = mlp.forward(small["mlp"], dims, enc)
    _, gy = mlp.mse(yy, tgt)
    abs_mlp, abs_denc = mlp.backward(np.abs(small["mlp"]), dims, [np.abs(x) for x in a],
                                     [np.where(x > 0, 1.0, -1.0) for x in z], np.abs(gy))
    _, g_abs = encode.encode_backward(lv, b, c, abs_denc, F)
    got = _table_grad(model, info)
    assert (np.abs(got[rows] - g_rows) <= 1e-4 * g_abs + 1e-12).all()
    untouched = np.ones(got.shape[0], bool)
    untouched[rows] = False
    assert (got[untouched] == 0).all()

    torch_g = np.concatenate([np.concatenate([l.weight.grad.cpu().numpy().ravel(), l.bias.grad.cpu().numpy()])
                              for l in net if isinstance(l, t.nn.Linear)])
    assert (np.abs(torch_g - g_mlp) <= 1e-4 * abs_mlp + 1e-12).all()
    assert encoder.anchor.grad is None
