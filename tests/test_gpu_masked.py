"""Masked compact tables (FHASH_LAYOUT_MASKED: rows only for the vertices near the dilated feature, the
irregular grids of Section 3.1's feature-only coreset) on the GPU, against the oracle and against the
rectangular Eq. 9 layout.

The level sizes (3x5x2x1, 6x9x7x2, 13x10x17x3, 30x27x31x8) cover R == 1 on time, R above and below
the FBB size and the finest level on the data grid.  Checked:
- active-vertex bits of every level and the compact bases bit-exact against the oracle;
- corner rows from fhash_lookup bit-exact (UINT64_MAX for inactive corners) at random points and at
  points on the faces of voxel footprints;
- encoding, float32 forward, loss, MLP and table gradients against the oracle within the bounds of
  the rectangular-layout tests; rows outside the batch's corners exactly zero;
- equivalence: a masked model holding the rectangular model's values at its active vertices gives
  bit-identical outputs at footprint points, a bit-identical rendered image (every rendered sample
  lies in a footprint) and the same first coreset-training loss;
- no mask: every vertex active and the rows are Eq. 9's;
- a checkpoint reloads the directories; bf16 and the allocation-free entry point are refused.
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import coreset, encode, index, masked, mlp, schedule, train

from _util import fh, read, set_params, to_dev, torch

pytestmark = pytest.mark.gpu
RES = [[3, 5, 2, 1], [6, 9, 7, 2], [13, 10, 17, 3], [30, 27, 31, 8]]
W = dict(workloads.SMALL, schedule=dict(mode="explicit", res=RES))
U64_MAX = np.uint64(0xFFFFFFFFFFFFFFFF)


def _build(mask, layout, dtype=0, seed=7):
    nx, ny, nz, nt = W["dims"]
    return fh().fhash_build(nx, ny, nz, nt, mask=mask, schedule=fh().make_schedule(**W["schedule"]), F=W["F"],
                            dtype=dtype, mlp_hidden_layers=W["hidden"], mlp_width=W["width"], seed=seed,
                            init_range=W["init_range"], layout=layout)


@pytest.fixture(scope="module")
def scene():
    f, m = workloads.make_field_and_mask(W)
    d = index.dilate(m)
    lo, size = index.fbb(d)
    dil = masked.fbb_mask(d, lo, size)
    lay = masked.MaskedLayout(RES, dil)
    model = _build(m, fh().LAYOUT_MASKED)
    info = fh().fhash_get_info(model)
    return dict(field=f, mask=m, dil=dil, lay=lay, model=model, info=info)


def _points(scene, n, seed):
    rs = np.random.default_rng(seed)
    c = rs.uniform(0, 1, (n, 4)).astype(np.float32)
    c[:3] = [[0, 0, 0, 0], [1, 1, 1, 1], [0.99, 0.51, 0.26, 0.74]]
    return np.concatenate([c, masked.footprint_points(scene["dil"], n, seed + 1),
                           masked.footprint_points(scene["dil"], n, seed + 2, edge=True)])


def _bits(active):
    """Active grid [Rt][Rz][Ry][Rx] -> little-endian 64-bit words of its Eq. 9 order."""
    flat = active.reshape(-1)
    pad = np.zeros((flat.size + 63) // 64 * 64, np.uint8)
    pad[:flat.size] = flat
    return np.packbits(pad, bitorder="little").view(np.uint64)


def test_active_bits_bases_and_rows_bit_exact(scene):
    info, lay, model = scene["info"], scene["lay"], scene["model"]
    assert info["res"] == RES
    assert info["total_rows"] == lay.rows_total < schedule.bases(RES)[1]
    assert list(info["base"][:len(RES)]) == lay.bases
    for l, R in enumerate(RES):
        want = _bits(masked.active_grid(scene["dil"], R))
        got = np.empty(want.size, np.uint64)
        fh().fhash_read_active(model, l, 0, got)
        assert np.array_equal(got, want), l
    c = _points(scene, 3000, 1)
    rows = torch().empty((c.shape[0], len(RES), 16), dtype=torch().int64, device="cuda")
    fh().fhash_lookup(model, to_dev(c), rows)
    rows = rows.cpu().numpy().view(np.uint64)
    for l, R in enumerate(RES):
        r_o, _ = encode.level_corners(c, R, lay.bases[l], lay.level(l))
        want = np.where(r_o >= 0, r_o.astype(np.uint64), U64_MAX)
        assert np.array_equal(rows[:, l, :], want), l
    assert (rows[3000:] != U64_MAX).all()  # footprint points see active corners only
    assert (rows[:3000] == U64_MAX).any()  # and some random points do not


def test_encode_forward_and_gradients(scene):
    info, lay, model = scene["info"], scene["lay"], scene["model"]
    F, dims = info["F"], info["mlp_dims"]
    table = synth.uniform(13, 50, info["n_table_params"], -0.5, 0.5)
    p = synth.init_mlp(13, dims)
    set_params(model, table, p)
    T = table.reshape(-1, F).astype(np.float64)
    c = _points(scene, 1500, 2)
    enc = torch().empty((c.shape[0], info["n_levels"] * F), dtype=torch().float32, device="cuda")
    fh().fhash_encode(model, to_dev(c), enc)
    ref = encode.encode(RES, lay.bases, c, T, lay)
    scale = encode.encode(RES, lay.bases, c, np.abs(T), lay)
    assert (np.abs(enc.cpu().numpy() - ref) <= 1e-5 * scale + 1e-30).all()
    out = torch().empty(c.shape[0], dtype=torch().float32, device="cuda")
    fh().fhash_forward(model, to_dev(c), out)
    y = mlp.forward(p, dims, ref)[0]
    assert (np.abs(out.cpu().numpy() - y) <= 1e-4 * np.maximum(np.abs(y), np.sqrt(np.mean(y ** 2)))).all()

    tgt = synth.sample(scene["field"], info["fbb_lo"], info["fbb_size"], c)
    loss = np.zeros(1, np.float64)
    fh().fhash_compute_grads(model, to_dev(c), to_dev(tgt), loss)
    L, _, g_mlp, (rows, g_rows) = train.loss_and_grads(RES, lay.bases, F, dims, T, p, c, tgt, lay)
    assert abs(loss[0] - L) <= 1e-5 * L
    n_t = info["n_table_params"]
    g = read(model, fh().STATE_GRAD, 0, n_t + info["n_mlp_params"]).astype(np.float64)
    yy, a, z = mlp.forward(p, dims, ref)
    _, gy = mlp.mse(yy, tgt)
    abs_mlp, abs_denc = mlp.backward(np.abs(p), dims, [np.abs(x) for x in a], [np.where(x > 0, 1.0, -1.0) for x in z],
                                     np.abs(gy))
    assert (np.abs(g[n_t:] - g_mlp) <= 1e-4 * abs_mlp + 1e-12).all()
    _, g_abs = encode.encode_backward(RES, lay.bases, c, abs_denc, F, lay)
    gt = g[:n_t].reshape(-1, F)
    assert (np.abs(gt[rows] - g_rows) <= 1e-4 * g_abs + 1e-12).all()
    untouched = np.ones(gt.shape[0], bool)
    untouched[rows] = False
    assert (gt[untouched] == 0).all()
    fh().fhash_apply_adam(model, W["adam"])
    fh().fhash_check(model)


def test_equivalence_with_the_rectangular_layout(scene, tmp_path):
    info, lay = scene["info"], scene["lay"]
    F = info["F"]
    lin = _build(scene["mask"], fh().LAYOUT_LINEAR)
    msk = _build(scene["mask"], fh().LAYOUT_MASKED)
    b, total = schedule.bases(RES)
    t_lin = synth.uniform(14, 50, total * F, -0.6, 0.6).reshape(-1, F)
    t_msk = np.zeros((lay.rows_total, F), np.float32)
    for l in range(len(RES)):
        r = lay.level(l).rank
        idx = np.flatnonzero(r >= 0)
        t_msk[r[idx]] = t_lin[b[l] + idx]
    p = synth.init_mlp(14, info["mlp_dims"])
    p[-1] = 0.45
    set_params(lin, t_lin, p)
    set_params(msk, t_msk, p)
    c = to_dev(np.concatenate([masked.footprint_points(scene["dil"], 20000, 21),
                               masked.footprint_points(scene["dil"], 5000, 22, edge=True)]))
    outs = []
    for model in (lin, msk):
        o = torch().empty(c.shape[0], dtype=torch().float32, device="cuda")
        fh().fhash_forward(model, c, o)
        outs.append(o.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    w, h = 40, 32
    tf = to_dev(synth.transfer_function(0.5))
    for t_norm in (0.35, 0.5):
        cam = synth.camera(synth.sphere_eye(9, 4), w, h)
        imgs = []
        for model in (lin, msk):
            rgba = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
            fh().fhash_render(model, cam, t_norm, tf, w, h, rgba)
            imgs.append(rgba.cpu().numpy())
        assert np.array_equal(imgs[0], imgs[1]) and imgs[0][..., 3].max() > 0
    # coreset training: every coreset sample sees active corners only, so the first loss is the same
    keys = [0, 3, 7]
    n_cs = [fh().fhash_coreset_build(model, scene["field"], keys) for model in (lin, msk)]
    assert n_cs[0] == n_cs[1] > 0
    hp = tuple(float(np.float32(x)) for x in W["adam"])
    losses = []
    for model in (lin, msk):
        loss = np.zeros(1, np.float64)
        fh().fhash_coreset_train_step(model, 5, 0, 0, 4096, hp, loss)
        losses.append(loss[0])
    assert losses[0] == losses[1]
    # the masked model keeps its directories through a checkpoint
    path = str(tmp_path / "masked.fhc")
    fh().fhash_save(msk, path)
    again = fh().fhash_load(path)
    assert fh().fhash_get_info(again)["total_rows"] == lay.rows_total
    for model in (msk, again):
        o = torch().empty(c.shape[0], dtype=torch().float32, device="cuda")
        fh().fhash_forward(model, c, o)
        outs.append(o.cpu().numpy())
    assert np.array_equal(outs[2], outs[3])
    got = np.empty((RES[-1][0] * RES[-1][1] * RES[-1][2] * RES[-1][3] + 63) // 64, np.uint64)
    fh().fhash_read_active(again, len(RES) - 1, 0, got)
    assert np.array_equal(got, _bits(masked.active_grid(scene["dil"], RES[-1])))
    fh().fhash_check(msk)


def test_no_mask_keeps_every_vertex():
    model = _build(None, fh().LAYOUT_MASKED)
    info = fh().fhash_get_info(model)
    b, total = schedule.bases(RES)
    assert info["total_rows"] == total and list(info["base"][:len(RES)]) == b
    lin = _build(None, fh().LAYOUT_LINEAR)
    c = to_dev(synth.coords(5, 2000))
    rows = [torch().empty((2000, len(RES), 16), dtype=torch().int64, device="cuda") for _ in range(2)]
    fh().fhash_lookup(model, c, rows[0])
    fh().fhash_lookup(lin, c, rows[1])
    assert torch().equal(rows[0], rows[1])


def test_refusals(scene):
    with pytest.raises(fh().FHashError):
        _build(scene["mask"], fh().LAYOUT_MASKED, dtype=fh().BF16)
    with pytest.raises(fh().FHashError):
        c = to_dev(synth.coords(6, 64))
        fh().fhash_compute_grads_noalloc(scene["model"], c, to_dev(np.zeros(64, np.float32)))
    lin = _build(scene["mask"], fh().LAYOUT_LINEAR)
    with pytest.raises(fh().FHashError):
        fh().fhash_read_active(lin, 0, 0, np.empty(1, np.uint64))
    with pytest.raises(fh().FHashError):
        fh().fhash_read_active(scene["model"], 0, 0, np.empty(10 ** 6, np.uint64))
