"""Several features in one model (fhash_build_desc.masks; Section 3.1 merges the occupancy grids of several
features for rendering), on the GPU against the oracle's merge (oracle/index.merge_features).

Features of the SMALL field: the blob cores (v > 0.8), a thin shell around them (0.30 < v < 0.33) and a
sparse random set of voxels.  With K = 2 and 3 features:
- the Feature Bounding Box and the occupancy grid of every time step are bit-exact;
- a masked-table model (FHASH_LAYOUT_MASKED) keeps exactly the oracle's active vertices of the union;
- a rendered image of the merged model matches the oracle's render over the merged occupancy (the
  tolerances of the single-feature render test: composited-sample counts equal on >= 99.9% of pixels,
  matched pixels within 2e-4, PSNR >= 60 dB);
- one feature given through masks[] builds the same model as through mask; mask and masks together are
  refused.
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import index, masked, render

from _util import fh, set_params, to_dev, torch

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


@pytest.fixture(scope="module")
def features():
    f, _ = workloads.make_field_and_mask(W1)
    core = synth.mask(f, 0.8)
    shell = synth.mask(f, 0.30, 0.33)
    rnd = (np.random.default_rng(8).random(f.shape) < 2e-4).astype(np.uint8)
    return f, [core, shell, rnd]


def _build(masks, layout=0, seed=3):
    nx, ny, nz, nt = W1["dims"]
    return fh().fhash_build(nx, ny, nz, nt, masks=masks, schedule=fh().make_schedule(**W1["schedule"]), F=W1["F"],
                            mlp_hidden_layers=W1["hidden"], mlp_width=W1["width"], seed=seed,
                            init_range=W1["init_range"], layout=layout)


@pytest.mark.parametrize("k", [2, 3])
def test_merged_fbb_and_occupancy(features, k):
    f, ms = features
    model = _build(ms[:k])
    info = fh().fhash_get_info(model)
    d = index.merge_features(ms[:k])
    lo, size = index.fbb(d)
    assert info["fbb_lo"] == lo and info["fbb_size"] == size
    occ = index.occupancy(d, lo, size)
    one = index.occupancy(index.dilate(ms[0]), lo, size)
    assert occ.sum() > one.sum()  # the other features add voxels
    for t in range(W1["dims"][3]):
        got = np.empty((size[2], size[1], size[0]), np.uint8)
        fh().fhash_read_occupancy(model, t, got)
        assert np.array_equal(got.astype(bool), occ[t]), t
    fh().fhash_check(model)


def test_merged_masked_layout(features):
    f, ms = features
    model = _build(ms, layout=fh().LAYOUT_MASKED)
    info = fh().fhash_get_info(model)
    d = index.merge_features(ms)
    lo, size = index.fbb(d)
    lay = masked.MaskedLayout(info["res"], masked.fbb_mask(d, lo, size))
    assert list(info["base"][:len(info["res"])]) == lay.bases and info["total_rows"] == lay.rows_total
    for l, R in enumerate(info["res"]):
        flat = masked.active_grid(masked.fbb_mask(d, lo, size), R).reshape(-1)
        pad = np.zeros((flat.size + 63) // 64 * 64, np.uint8)
        pad[:flat.size] = flat
        want = np.packbits(pad, bitorder="little").view(np.uint64)
        got = np.empty(want.size, np.uint64)
        fh().fhash_read_active(model, l, 0, got)
        assert np.array_equal(got, want), l


def test_merged_render_parity(features):
    f, ms = features
    model = _build(ms)
    info = fh().fhash_get_info(model)
    table = synth.uniform(23, 50, info["n_table_params"], -0.6, 0.6)
    p = synth.init_mlp(23, info["mlp_dims"])
    p[-1] = 0.45
    set_params(model, table, p)
    d = index.merge_features(ms)
    occ = index.occupancy(d, info["fbb_lo"], info["fbb_size"])
    ev = render.model_eval_fn(info["res"], info["base"], table.reshape(-1, info["F"]).astype(np.float64),
                              p.astype(np.float64), info["mlp_dims"])
    w, h, t = 56, 40, 0.35
    cam = synth.camera(synth.sphere_eye(12, 1), w, h)
    tf = synth.transfer_function(0.5)
    rgba = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
    cnt = torch().empty((h, w), dtype=torch().int32, device="cuda")
    fh().fhash_render(model, cam, t, to_dev(tf), w, h, rgba, cnt)
    img, c = rgba.cpu().numpy(), cnt.cpu().numpy()
    ref, rc = render.render(ev, cam, w, h, info["fbb_size"], occ, np.float32(t), tf)
    same = c == rc
    assert rc.sum() > 0 and same.mean() >= 0.999, same.mean()
    assert np.abs(img[same] - ref[same]).max() <= 2e-4
    mse = np.mean((img - ref) ** 2)
    assert mse == 0 or 10 * np.log10(1.0 / mse) >= 60


def test_single_feature_list_and_refusal(features):
    f, ms = features
    a = _build(ms[:1])
    nx, ny, nz, nt = W1["dims"]
    b = fh().fhash_build(nx, ny, nz, nt, mask=ms[0], schedule=fh().make_schedule(**W1["schedule"]), F=W1["F"],
                         mlp_hidden_layers=W1["hidden"], mlp_width=W1["width"], seed=3, init_range=W1["init_range"])
    ia, ib = fh().fhash_get_info(a), fh().fhash_get_info(b)
    assert ia["fbb_lo"] == ib["fbb_lo"] and ia["fbb_size"] == ib["fbb_size"] and ia["res"] == ib["res"]
    for t in (0, 5):
        sz = ia["fbb_size"]
        oa, ob = (np.empty((sz[2], sz[1], sz[0]), np.uint8) for _ in range(2))
        fh().fhash_read_occupancy(a, t, oa)
        fh().fhash_read_occupancy(b, t, ob)
        assert np.array_equal(oa, ob)
    with pytest.raises(fh().FHashError) as e:
        fh().fhash_build(nx, ny, nz, nt, mask=ms[0], masks=ms[1:], schedule=fh().make_schedule(**W1["schedule"]),
                         F=W1["F"], mlp_hidden_layers=W1["hidden"], mlp_width=W1["width"])
    assert e.value.status == 1
