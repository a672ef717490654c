"""What the learned part gains (GPU).

A small F-Hash model (8 levels, geometric 4^3x2 -> 32^3x8, F=2, MLP 2x64: about 0.6 M parameters) is
trained by the library's own kernels (fhash_train_step, Adam lr 1e-2) on the advect-128^3x32 field
(67 M voxels, so the model is about 100x smaller than the data).  Then its PSNR on 2^18 held-out
points is compared with:
(i)  the same model untrained (the initial tables and MLP);
(ii) the method without a network: the field sampled on a plain vertex-aligned 4D grid over the
     Feature Bounding Box with at least as many values as the model has parameters, interpolated
     quadrilinearly (Eqs. 10-12 on a single level, with the oracle's interpolation).
PSNR = 10 log10(range^2 / MSE), range = max - min of the held-out targets.  The test prints every
number and requires the trained model to gain at least 10 dB over (i) and to beat (ii).  Measured on a
GB300: 48.3 dB trained, 13.3 dB untrained, 43.5 dB for the 43x43x43x11 grid (874,577 values against
809,847 parameters).
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import encode

from _util import build, fh, to_dev, torch

pytestmark = pytest.mark.gpu
W = dict(workloads.MEDIUM, name="advect-128^3x32 small model", hidden=2, width=64,
         schedule=dict(mode="geometric", n_levels=8, r0=[4, 4, 4, 2], r1=[32, 32, 32, 8]))
STEPS, BATCH, N_EVAL = 600, 1 << 16, 1 << 18


def _psnr(pred, ref):
    mse = float(np.mean((pred.astype(np.float64) - ref) ** 2))
    rng = float(ref.max() - ref.min())
    return 10 * np.log10(rng * rng / mse)


def _grid_baseline(field, lo, size, n_params, pts):
    S = np.array(list(size) + [field.shape[0]], np.float64)  # FBB extent in x, y, z and the time steps
    s = (n_params / S.prod()) ** 0.25
    while True:
        g = np.maximum(2, np.ceil(s * S)).astype(np.int64)
        if g.prod() >= n_params:
            break
        s *= 1.01
    axes = [np.arange(k, dtype=np.float64) / (k - 1) for k in g]
    tt, zz, yy, xx = np.meshgrid(axes[3], axes[2], axes[1], axes[0], indexing="ij")
    verts = np.stack([xx.ravel(), yy.ravel(), zz.ravel(), tt.ravel()], 1).astype(np.float32)
    values = synth.sample(field, lo, size, verts).astype(np.float64)[:, None]  # row = Eq. 9 order
    pred = encode.interpolate_level(pts, [int(k) for k in g], 0, values)[:, 0]
    return pred, [int(k) for k in g]


def test_trained_network_gain(capsys):
    field, mask = workloads.make_field_and_mask(W)
    model = build(W, mask=mask, seed=11)
    info = fh().fhash_get_info(model)
    lo, size = info["fbb_lo"], info["fbb_size"]
    n_params = info["n_table_params"] + info["n_mlp_params"]

    pts = synth.coords(900, N_EVAL)
    ref = synth.sample(field, lo, size, pts).astype(np.float64)
    out = torch().empty(N_EVAL, dtype=torch().float32, device="cuda")
    dpts = to_dev(pts)

    def model_psnr():
        fh().fhash_forward(model, dpts, out)
        return _psnr(out.cpu().numpy(), ref)

    p_untrained = model_psnr()
    for k in range(STEPS):
        c = synth.coords(1000 + k, BATCH)
        fh().fhash_train_step(model, to_dev(c), to_dev(synth.sample(field, lo, size, c)), W["adam"])
    p_trained = model_psnr()
    grid_pred, g = _grid_baseline(field, lo, size, n_params, pts)
    p_grid = _psnr(grid_pred, ref)
    with capsys.disabled():
        print("\nlearned part: %d parameters; PSNR trained %.2f dB | untrained %.2f dB | plain grid %s "
              "(%d values) %.2f dB" % (n_params, p_trained, p_untrained, "x".join(map(str, g)), int(np.prod(g)),
                                       p_grid))
    assert np.isfinite([p_trained, p_untrained, p_grid]).all()
    assert p_trained >= p_untrained + 10.0
    assert p_trained > p_grid
