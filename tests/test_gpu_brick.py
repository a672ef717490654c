"""The brick row layout (FHASH_LAYOUT_BRICK: 4x4x4 bricks per time slice, a linearisation Section 3.2.3
allows in place of Eq. 9) on the GPU, against the oracle and against the linear layout.

The level sizes (3x5x2x1, 6x9x7x2, 13x10x17x3, 30x27x31x8) are not multiples of 4, so every level
has partial bricks.  Checked:
- corner rows from fhash_lookup bit-exact against the oracle's brick rows;
- encoding within 1e-5 x sum |w T|, float32 forward within 1e-4 x max(|o|, RMS(o)), loss, MLP and
  table gradients within the term-magnitude bounds of the linear-layout tests;
- relabelling: a brick model holding the linear model's vertex values at its own rows gives
  bit-identical outputs in float32, in the bf16 fused and split paths, and in a rendered image;
- a checkpoint of a brick model reloads with its layout.
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import encode, mlp, train

from _util import fh, read, set_params, to_dev, torch

pytestmark = pytest.mark.gpu
RES = [[3, 5, 2, 1], [6, 9, 7, 2], [13, 10, 17, 3], [30, 27, 31, 8]]
W = dict(workloads.SMALL, schedule=dict(mode="explicit", res=RES))


def _build(mask, layout, dtype=0, seed=7):
    nx, ny, nz, nt = W["dims"]
    return fh().fhash_build(nx, ny, nz, nt, mask=mask, schedule=fh().make_schedule(**W["schedule"]), F=W["F"],
                            dtype=dtype, mlp_hidden_layers=W["hidden"], mlp_width=W["width"], seed=seed,
                            init_range=W["init_range"], layout=layout)


@pytest.fixture(scope="module")
def scene():
    f, m = workloads.make_field_and_mask(W)
    brk = _build(m, fh().LAYOUT_BRICK)
    info = fh().fhash_get_info(brk)
    assert info["res"] == RES
    return dict(field=f, mask=m, brk=brk, info=info)


def _coords(n, seed):
    c = synth.coords(seed, n)
    c[:3] = [[0, 0, 0, 0], [1, 1, 1, 1], [0.99, 0.51, 0.26, 0.74]]
    return c


def _relabel(info, t_lin):
    """Table of a brick model holding, for every vertex, the value the linear table holds for it."""
    t_brk = np.empty_like(t_lin)
    for R, b in zip(info["res"], info["base"]):
        Rx, Ry, Rz, Rt = R
        t, z, y, x = (a.ravel() for a in np.meshgrid(*[np.arange(k) for k in (Rt, Rz, Ry, Rx)], indexing="ij"))
        t_brk[b + encode.fhash(t, x, y, z, R, "brick")] = t_lin[b + encode.fhash(t, x, y, z, R)]
    return t_brk


def test_brick_lookup_rows_bit_exact(scene):
    info = scene["info"]
    c = _coords(3001, 1)
    L = info["n_levels"]
    rows = torch().empty((c.shape[0], L, 16), dtype=torch().int64, device="cuda")
    fh().fhash_lookup(scene["brk"], to_dev(c), rows)
    rows = rows.cpu().numpy().view(np.uint64)
    for l in range(L):
        r_o, _ = encode.level_corners(c, info["res"][l], info["base"][l], "brick")
        assert np.array_equal(rows[:, l, :], r_o.astype(np.uint64)), l


def test_brick_encode_forward_and_gradients(scene):
    info, model = scene["info"], scene["brk"]
    lv, b, F, dims = info["res"], info["base"], info["F"], info["mlp_dims"]
    table = synth.uniform(13, 50, info["n_table_params"], -0.5, 0.5)
    p = synth.init_mlp(13, dims)
    set_params(model, table, p)
    T = table.reshape(-1, F).astype(np.float64)
    c = _coords(4099, 2)
    enc = torch().empty((c.shape[0], info["n_levels"] * F), dtype=torch().float32, device="cuda")
    fh().fhash_encode(model, to_dev(c), enc)
    ref = encode.encode(lv, b, c, T, "brick")
    scale = encode.encode(lv, b, c, np.abs(T), "brick")
    assert (np.abs(enc.cpu().numpy() - ref) <= 1e-5 * scale + 1e-30).all()
    out = torch().empty(c.shape[0], dtype=torch().float32, device="cuda")
    fh().fhash_forward(model, to_dev(c), out)
    y = mlp.forward(p, dims, ref)[0]
    assert (np.abs(out.cpu().numpy() - y) <= 1e-4 * np.maximum(np.abs(y), np.sqrt(np.mean(y ** 2)))).all()

    tgt = synth.sample(scene["field"], info["fbb_lo"], info["fbb_size"], c)
    loss = np.zeros(1, np.float64)
    fh().fhash_compute_grads(model, to_dev(c), to_dev(tgt), loss)
    L, _, g_mlp, (rows, g_rows) = train.loss_and_grads(lv, b, F, dims, T, p, c, tgt, "brick")
    assert abs(loss[0] - L) <= 1e-5 * L
    n_t = info["n_table_params"]
    g = read(model, fh().STATE_GRAD, 0, n_t + info["n_mlp_params"]).astype(np.float64)
    yy, a, z = mlp.forward(p, dims, ref)
    _, gy = mlp.mse(yy, tgt)
    abs_mlp, abs_denc = mlp.backward(np.abs(p), dims, [np.abs(x) for x in a], [np.where(x > 0, 1.0, -1.0) for x in z],
                                     np.abs(gy))
    assert (np.abs(g[n_t:] - g_mlp) <= 1e-4 * abs_mlp + 1e-12).all()
    _, g_abs = encode.encode_backward(lv, b, c, abs_denc, F, "brick")
    gt = g[:n_t].reshape(-1, F)
    assert (np.abs(gt[rows] - g_rows) <= 1e-4 * g_abs + 1e-12).all()
    untouched = np.ones(gt.shape[0], bool)
    untouched[rows] = False
    assert (gt[untouched] == 0).all()
    fh().fhash_apply_adam(model, W["adam"])
    fh().fhash_check(model)


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_brick_is_a_relabelling_bit_identical(scene, dtype, tmp_path):
    info = scene["info"]
    dt = fh().FP32 if dtype == "fp32" else fh().BF16
    lin = _build(scene["mask"], fh().LAYOUT_LINEAR, dt)
    brk = _build(scene["mask"], fh().LAYOUT_BRICK, dt)
    t_lin = synth.uniform(14, 50, info["n_table_params"], -0.6, 0.6).reshape(-1, info["F"])
    p = synth.init_mlp(14, info["mlp_dims"])
    p[-1] = 0.45
    set_params(lin, t_lin, p)
    set_params(brk, _relabel(info, t_lin), p)
    c = to_dev(_coords(20000, 3))
    outs = []
    paths = [None] if dtype == "fp32" else [fh().FORWARD_FUSED, fh().FORWARD_SPLIT]
    for model in (lin, brk):
        for path in paths:
            if path is not None:
                fh().fhash_set_forward_path(model, path)
            o = torch().empty(c.shape[0], dtype=torch().float32, device="cuda")
            fh().fhash_forward(model, c, o)
            outs.append(o.cpu().numpy())
    half = len(outs) // 2
    for a, b in zip(outs[:half], outs[half:]):
        assert np.array_equal(a, b)
    w, h = 40, 32
    cam = synth.camera(synth.sphere_eye(9, 4), w, h)
    tf = to_dev(synth.transfer_function(0.5))
    imgs = []
    for model in (lin, brk):
        rgba = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
        fh().fhash_render(model, cam, 0.35, tf, w, h, rgba)
        imgs.append(rgba.cpu().numpy())
    assert np.array_equal(imgs[0], imgs[1]) and imgs[0][..., 3].max() > 0
    # a checkpoint keeps the layout
    path = str(tmp_path / "brick.fhc")
    fh().fhash_save(brk, path)
    again = fh().fhash_load(path)
    o = torch().empty(c.shape[0], dtype=torch().float32, device="cuda")
    fh().fhash_forward(again, c, o)
    assert np.array_equal(o.cpu().numpy(), outs[half])
    fh().fhash_check(brk)
