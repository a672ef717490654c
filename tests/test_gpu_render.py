"""GPU parity of the ARM renderer (Section 3.3, Algorithm 1) and the time-slice decode against the oracle.

Parameters are seeded inputs (synth), written into the model through the C ABI; the oracle evaluates
the same parameters in float64.  Tolerances: per-pixel composited sample counts equal on >= 99.9% of
pixels (float32 vs float64 values can move the 0.99 opacity cut by one sample); pixels whose counts
match within 2e-4 absolute in every channel; image PSNR vs the oracle >= 60 dB; the image is
bit-identical for pace limits 1 and 64 (the pace changes batching, not samples).  With a transfer function
of zero opacity no ray stops early, so every pixel's composited-sample count is the number of occupied
samples on its ray: it must equal the oracle's exactly, which pins the empty-space skipping (8^3
bricks, 4^3 and 2^3 sub-blocks) to skipping unoccupied samples only.
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import encode, index, mlp, render

from _util import build, fh, set_params, to_dev, torch

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


@pytest.fixture(scope="module")
def scene():
    f, m = workloads.make_field_and_mask(W1)
    model = build(W1, mask=m)
    info = fh().fhash_get_info(model)
    table = synth.uniform(21, 50, info["n_table_params"], -0.6, 0.6)
    p = synth.init_mlp(21, info["mlp_dims"])
    p[-1] = 0.45  # output bias: values around the middle of the transfer function
    set_params(model, table, p)
    d = index.dilate(m)
    occ = index.occupancy(d, info["fbb_lo"], info["fbb_size"])
    T = table.reshape(-1, info["F"]).astype(np.float64)
    ev = render.model_eval_fn(info["res"], info["base"], T, p.astype(np.float64), info["mlp_dims"])
    return dict(model=model, info=info, occ=occ, eval=ev, table=T, p=p)


def _render_gpu(sc, cam, t, w, h, pace=64):
    tf = synth.transfer_function(0.5)
    rgba = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
    cnt = torch().empty((h, w), dtype=torch().int32, device="cuda")
    st = fh().fhash_render(sc["model"], cam, t, to_dev(tf), w, h, rgba, cnt, max_pace=pace)
    return rgba.cpu().numpy(), cnt.cpu().numpy(), st, tf


@pytest.mark.parametrize("view,t", [(0, 0.0), (1, 0.3), (2, 1.0)])
def test_render_parity(scene, view, t):
    w, h = 64, 48
    cam = synth.camera(synth.sphere_eye(5, view), w, h)
    img, cnt, st, tf = _render_gpu(scene, cam, t, w, h)
    ref, rcnt = render.render(scene["eval"], cam, w, h, scene["info"]["fbb_size"], scene["occ"], np.float32(t), tf)
    same = cnt == rcnt
    assert same.mean() >= 0.999, (same.mean(), int((~same).sum()))
    assert rcnt.sum() > 0
    assert np.abs(img[same] - ref[same]).max() <= 2e-4
    mse = np.mean((img - ref) ** 2)
    assert mse == 0 or 10 * np.log10(1.0 / mse) >= 60
    assert st["samples_composited"] == cnt.sum() and st["rounds"] >= 1


def test_pace_invariance(scene):
    w, h = 40, 40
    cam = synth.camera(synth.sphere_eye(5, 3), w, h)
    a, ca, sa, _ = _render_gpu(scene, cam, 0.6, w, h, pace=64)
    b, cb, sb, _ = _render_gpu(scene, cam, 0.6, w, h, pace=1)
    assert np.array_equal(a, b) and np.array_equal(ca, cb)
    assert sb["rounds"] > sa["rounds"]


def test_decode_parity(scene):
    info = scene["info"]
    for up, t in ((1, 0.0), (2, 0.37)):
        dims = fh().fhash_decode_dims(scene["model"], up)
        out = torch().empty((dims[2], dims[1], dims[0]), dtype=torch().float32, device="cuda")
        fh().fhash_decode(scene["model"], t, up, out)
        u, shape = render.decode_coords(info["fbb_size"], up, np.float32(t))
        assert list(shape) == [dims[2], dims[1], dims[0]]
        ref = scene["eval"](u).reshape(shape)
        got = out.cpu().numpy()
        tol = 1e-4 * np.maximum(np.abs(ref), np.sqrt(np.mean(ref ** 2)))
        assert (np.abs(got - ref) <= tol).all(), np.abs(got - ref).max()


@pytest.mark.parametrize("view,t", [(0, 0.0), (4, 0.43), (6, 1.0), (7, 0.5)])
def test_skipping_keeps_every_occupied_sample(scene, view, t):
    w, h = 80, 60
    cam = synth.camera(synth.sphere_eye(11, view), w, h)
    tf = synth.transfer_function(0.5)
    tf[:, 3] = 0.0
    rgba = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
    cnt = torch().empty((h, w), dtype=torch().int32, device="cuda")
    st = fh().fhash_render(scene["model"], cam, t, to_dev(tf), w, h, rgba, cnt)
    _, rcnt = render.render(scene["eval"], cam, w, h, scene["info"]["fbb_size"], scene["occ"], np.float32(t), tf)
    got = cnt.cpu().numpy()
    assert rcnt.sum() > 1000
    assert np.array_equal(got, rcnt), int((got != rcnt).sum())
    # and the marcher visited fewer positions than the samples it would step through one by one
    assert st["steps_marched"] > 0
